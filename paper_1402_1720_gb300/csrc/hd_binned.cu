// Binned SC: SC as the paper ran it (Sec. 2.2 data cuts; Sec. 3.2, its
// implementation paragraphs).  Histories are binned by gantry angle and by
// the mid-point displacement of their path; per bin, 3 sigma cuts on WEPL
// and both slopes; a bin whose kept histories average below the WEPL cutoff
// is missed and its line is carved in every slice it covers; the carved
// image is averaged over a window in each slice and thresholded.
//
// Four stream-ordered kernels, all integer arithmetic:
//   binned_stats_kernel  one thread per history: 7 64-bit atomics into its
//                        bin's row of the table (n, S and Q of 3 values)
//   binned_cut_kernel    one thread per history: the 3 sigma test in 128-bit
//                        integers against the finished statistics, kept n
//                        and kept WEPL sum by 2 atomics
//   binned_carve_kernel  one block per (angle bin, slice): the lines of the
//                        block's missed bins walked run by run into a bitmap
//                        of the slice in shared memory, merged into the
//                        volume bitmap with one atomicAnd per changed word
//   binned_filter_kernel one thread per voxel: the window count of uncarved
//                        voxels, the hull byte and the carved byte
#include <cmath>
#include <new>

#include "hd_geom.cuh"

namespace hd {

struct BinQ {
    int n_ang, n_u, n_v, k;
    long long ang_q, u_q, v_q, u_lo_q, v_lo_q;  // Q16 degrees and mm
    long long miss_q8;                          // 1/256 mm
    int w, min_count;
};

namespace {

constexpr int kBinThreads = 256;
constexpr int kPassBlocksPerSm = 6;  // resident blocks of the per-history passes (40 registers)
constexpr int kCarveThreads = 192;
constexpr int kAccWords = 9;
constexpr int kCtrWords = 8;
constexpr int kMaxSmemWords = 48 * 1024;  // slice bitmaps up to 192 KB in shared memory
constexpr long long kFull = 360LL * 65536;

__device__ __forceinline__ long long q8_of(float x) { return __float2ll_rn(x * 256.0f); }

// Bin of one history, -1 when it is not binned; x receives WEPL, lateral and
// vertical slope in 1/256 mm.
__device__ __forceinline__ long long bin_of(const BinQ &b, float ang, float ui, float vi, float uo,
                                            float vo, float wepl, long long x[3])
{
    if (!(fabsf(ang) < 1048576.0f) || !(fabsf(wepl) < 1024.0f)) return -1;
    if (!(fabsf(ui) < 4096.0f) || !(fabsf(vi) < 4096.0f) || !(fabsf(uo) < 4096.0f) ||
        !(fabsf(vo) < 4096.0f))
        return -1;
    x[0] = q8_of(wepl);
    x[1] = q8_of(uo) - q8_of(ui);
    x[2] = q8_of(vo) - q8_of(vi);
    if (llabs(x[1]) >= 1024 * 256 || llabs(x[2]) >= 1024 * 256) return -1;
    long long a = q16_of(ang);  // |a| < 2^36: the quotients below are small
    a -= floordiv_small(a, kFull) * kFull;
    long long ia = floordiv_small(2 * a + b.ang_q, 2 * b.ang_q);  // nearest centre
    if (ia == b.n_ang) ia = 0;
    const long long u2 = q16_of(ui) + q16_of(uo), v2 = q16_of(vi) + q16_of(vo);
    const long long iu = floordiv_small(u2 - 2 * b.u_lo_q, 2 * b.u_q);
    const long long iv = floordiv_small(v2 - 2 * b.v_lo_q, 2 * b.v_q);
    if (iu < 0 || iu >= b.n_u || iv < 0 || iv >= b.n_v) return -1;
    return ia + static_cast<long long>(b.n_ang) * (iu + static_cast<long long>(b.n_u) * iv);
}

// x within k population standard deviations of a bin holding n values of
// sum S and sum of squares Q: (n x - S)^2 <= k^2 (n Q - S^2).
__device__ __forceinline__ bool within(long long n, long long S, long long Q, long long x, int k)
{
    const __int128 d = static_cast<__int128>(n) * x - S;
    const __int128 var_n2 = static_cast<__int128>(n) * Q - static_cast<__int128>(S) * S;
    return d * d <= static_cast<__int128>(k * k) * var_n2;
}

__device__ __forceinline__ bool bin_missed(const unsigned long long *a, long long miss_q8)
{
    const long long kn = static_cast<long long>(a[7]);
    const long long ks = static_cast<long long>(a[8]);
    return kn > 0 && ks < miss_q8 * kn;
}

__device__ __forceinline__ void warp_add(unsigned long long v, unsigned long long *dst)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0) atomicAdd(dst, v);
}

__global__ void __launch_bounds__(kBinThreads, kPassBlocksPerSm) binned_stats_kernel(Inputs in, int64_t n, BinQ b,
                                                                   unsigned long long *acc,
                                                                   unsigned long long *ctr)
{
    unsigned long long binned = 0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += stride) {
        long long x[3];
        const long long bi = bin_of(b, in.angle[i], in.u_in[i], in.v_in[i], in.u_out[i],
                                    in.v_out[i], in.wepl[i], x);
        if (bi < 0) continue;
        unsigned long long *a = acc + kAccWords * bi;
        atomicAdd(a, 1ull);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            atomicAdd(a + 1 + q, static_cast<unsigned long long>(x[q]));
            atomicAdd(a + 4 + q, static_cast<unsigned long long>(x[q] * x[q]));
        }
        ++binned;
    }
    warp_add(binned, ctr + 0);
}

// Reads words 0-6 of a bin row (fixed since the statistics phase ended)
// while other threads add to words 7 and 8.
__global__ void __launch_bounds__(kBinThreads, kPassBlocksPerSm) binned_cut_kernel(Inputs in, int64_t n, BinQ b,
                                                                 unsigned long long *acc,
                                                                 unsigned long long *ctr)
{
    unsigned long long cut = 0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += stride) {
        long long x[3];
        const long long bi = bin_of(b, in.angle[i], in.u_in[i], in.v_in[i], in.u_out[i],
                                    in.v_out[i], in.wepl[i], x);
        if (bi < 0) continue;
        unsigned long long *a = acc + kAccWords * bi;
        const long long cnt = static_cast<long long>(a[0]);
        bool keep = true;
#pragma unroll
        for (int q = 0; q < 3; ++q)
            keep = keep && within(cnt, static_cast<long long>(a[1 + q]),
                                  static_cast<long long>(a[4 + q]), x[q], b.k);
        if (!keep) {
            ++cut;
            continue;
        }
        atomicAdd(a + 7, 1ull);
        atomicAdd(a + 8, static_cast<unsigned long long>(x[0]));
    }
    warp_add(cut, ctr + 1);
}

__global__ void __launch_bounds__(kBinThreads) binned_bins_kernel(const unsigned long long *acc,
                                                                  int64_t nb, long long miss_q8,
                                                                  unsigned long long *ctr)
{
    unsigned long long used = 0, missed = 0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nb;
         i += stride) {
        const unsigned long long *a = acc + kAccWords * i;
        used += a[0] != 0 ? 1 : 0;
        missed += bin_missed(a, miss_q8) ? 1 : 0;
    }
    warp_add(used, ctr + 2);
    warp_add(missed, ctr + 3);
}

// Clears the bits of one run of a line in a slice bitmap (bit x + nx y,
// 1 = not carved).  An x-major run is a row segment, contiguous bits cleared
// a word at a time; a y-major run (row = x) is a column segment, one bit per
// voxel.  Runs come from a walk clipped to the slice, so they lie inside it;
// the checks only guard the bitmap.
__device__ __forceinline__ void clear_run(uint32_t *img, bool ymaj, int row, int lo, int hi,
                                          int nx, uint32_t plane)
{
    if (!ymaj) {
        const uint32_t l0 = static_cast<uint32_t>(row * nx + lo);
        const uint32_t l1 = static_cast<uint32_t>(row * nx + hi);
        if (l1 >= plane || l0 > l1) return;
        const uint32_t w0 = l0 >> 5, w1 = l1 >> 5;
        for (uint32_t w = w0; w <= w1; ++w) {
            const uint32_t a = w == w0 ? (l0 & 31u) : 0u;
            const uint32_t b = w == w1 ? (l1 & 31u) : 31u;
            const uint32_t m = b - a == 31u ? 0xffffffffu : ((1u << (b - a + 1u)) - 1u) << a;
            atomicAnd(img + w, ~m);
        }
    } else {
        for (int y = lo; y <= hi; ++y) {
            const uint32_t l = static_cast<uint32_t>(row + nx * y);
            if (l < plane) atomicAnd(img + (l >> 5), ~(1u << (l & 31u)));
        }
    }
}

// Host-computed line tables: centre angle of each angle bin, lateral centre
// of each u bin, centre height and vertical bin (or -1) of each slice.
struct LineTables {
    const float *ang_c, *u_c, *zc;
    const int *slice_bin;
};

constexpr int kMaxLinesPerBlock = 1024;  // lateral bins a block lists at once

// One block per (angle bin, slice): the block's missed bins are listed in
// shared memory, then each thread walks lines from the list.  A line lies at
// the slice's centre height, so its walk is clipped to the slice (a box one
// voxel deep) and is lean unless a crossing ties with another: the runs then
// come from the closed-form cursor, otherwise from the general run walk.
template <bool kShared>
__global__ void __launch_bounds__(kCarveThreads) binned_carve_kernel(
    const unsigned long long *acc, BinQ b, GeomQ g, Cordic cd, LineTables t, uint32_t *bits,
    int wps, unsigned long long *ctr)
{
    extern __shared__ uint32_t sm[];
    __shared__ int s_list[kMaxLinesPerBlock];
    __shared__ int s_warp[kCarveThreads / 32];
    __shared__ long long s_cs[2];
    const int ia = blockIdx.x, z = blockIdx.y;
    const int iv = t.slice_bin[z];
    if (iv < 0) return;  // the same for the whole block
    uint32_t *gimg = bits + static_cast<size_t>(z) * wps;
    uint32_t *img = kShared ? sm : gimg;
    if (kShared)
        for (int w = threadIdx.x; w < wps; w += blockDim.x) sm[w] = 0xffffffffu;
    const uint32_t plane = static_cast<uint32_t>(g.nx) * static_cast<uint32_t>(g.ny);
    const float zc = t.zc[z];
    if (threadIdx.x == 0) {  // the block's gantry cos and sin, once
        long long c, sn;
        cordic_cs(q16_of(t.ang_c[ia]), cd, c, sn);
        s_cs[0] = c;
        s_cs[1] = sn;
    }
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    unsigned long long lines = 0, outside = 0;
    for (int base = 0; base < b.n_u; base += kMaxLinesPerBlock) {
        // the chunk's missed bins, listed in lateral order (neighbouring
        // lanes then walk neighbouring, similar lines)
        const int end = min(b.n_u, base + kMaxLinesPerBlock);
        int nl = 0;
        for (int c0 = base; c0 < end; c0 += blockDim.x) {
            const int iu = c0 + static_cast<int>(threadIdx.x);
            bool miss = false;
            if (iu < end) {
                const long long bi = ia + static_cast<long long>(b.n_ang) *
                                              (iu + static_cast<long long>(b.n_u) * iv);
                miss = bin_missed(acc + kAccWords * bi, b.miss_q8);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, miss);
            if (lane == 0) s_warp[warp] = __popc(bal);
            __syncthreads();
            int off = nl, tot = 0;
            for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) {
                off += k < static_cast<int>(warp) ? s_warp[k] : 0;
                tot += s_warp[k];
            }
            if (miss) s_list[off + __popc(bal & ((1u << lane) - 1u))] = iu;
            nl += tot;
            __syncthreads();
        }
        const long long cs = s_cs[0], sn = s_cs[1];
        for (int j = threadIdx.x; j < nl; j += blockDim.x) {
            ++lines;
            const float lu = t.u_c[s_list[j]];
            int32_t r[6];
            if (!endpoints_cs(g, cs, sn, lu, zc, lu, zc, r)) {
                ++outside;
                continue;
            }
            const int32_t gi[3] = {r[0], r[1], r[2] - (z << 16)};
            const int32_t go[3] = {r[3], r[4], r[5] - (z << 16)};
            RunWalk w;
            if (!run_begin(w, gi, go, g.nx, g.ny, 1)) continue;
            const bool ymaj = (w.flags >> 5) & 1;
            LeanWalk L;
            int row, lo, hi;
            if (lean_of(w, L)) {
                uint32_t o[kLeanWords];
                lean_pack(L, o);
                LeanCursor c;
                if (!lean_start(o, 1, c)) continue;  // rows counted one by one
                unsigned ends = 0;
                bool more;
                do {
                    more = lean_run(c, row, lo, hi, ends);
                    clear_run(img, ymaj, row, lo, hi, g.nx, plane);
                } while (more);
            } else {
                while (run_next(w, row, lo, hi)) clear_run(img, ymaj, row, lo, hi, g.nx, plane);
            }
        }
        __syncthreads();  // the list is rebuilt next round
    }
    if (kShared) {
        for (int w = threadIdx.x; w < wps; w += blockDim.x) {
            const uint32_t m = sm[w];
            if (m != 0xffffffffu) atomicAnd(gimg + w, m);
        }
    }
    warp_add(lines, ctr + 4);
    warp_add(outside, ctr + 5);
}

// Window count of uncarved voxels in each slice (outside the grid counts as
// carved); hull = count >= min_count.
__global__ void __launch_bounds__(256) binned_filter_kernel(const uint32_t *bits, int wps, int nx,
                                                            int ny, int r, int min_count,
                                                            uint8_t *mask, uint8_t *carved)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const uint32_t *img = bits + static_cast<size_t>(z) * wps;
    auto bit = [&](int X, int Y) {
        const uint32_t l = static_cast<uint32_t>(X) + static_cast<uint32_t>(nx) * Y;
        return static_cast<int>((__ldg(img + (l >> 5)) >> (l & 31u)) & 1u);
    };
    int c = 0;
    for (int dy = -r; dy <= r; ++dy) {
        const int Y = y + dy;
        if (Y < 0 || Y >= ny) continue;
        for (int dx = -r; dx <= r; ++dx) {
            const int X = x + dx;
            if (X >= 0 && X < nx) c += bit(X, Y);
        }
    }
    const size_t v = static_cast<size_t>(x) + static_cast<size_t>(nx) * (y + static_cast<size_t>(ny) * z);
    mask[v] = c >= min_count ? 1 : 0;
    carved[v] = static_cast<uint8_t>(bit(x, y));
}

int grid_for(int64_t n, int sm_count, int per_sm = 8)
{
    int64_t blocks = (n + kBinThreads - 1) / kBinThreads;
    const int64_t cap = static_cast<int64_t>(sm_count > 0 ? sm_count : 1) * per_sm;
    if (blocks > cap) blocks = cap;
    return static_cast<int>(blocks < 1 ? 1 : blocks);
}

}  // namespace
}  // namespace hd

// ------------------------------------------------------------------ C ABI

struct hd_binned {
    int device = 0;
    int sm_count = 0;
    hd_geometry geom{};
    hd_binned_params params{};
    hd::GeomQ gq{};
    hd::Cordic cordic{};
    hd::BinQ bq{};
    int64_t V = 0;
    int64_t nb = 0;
    int wps = 0;  // bitmap words per slice
    unsigned long long *acc = nullptr;  // nb x 9
    unsigned long long *ctr = nullptr;  // 8 counters
    uint32_t *bits = nullptr;           // nz x wps carved bitmap (1 = not carved)
    uint8_t *mask = nullptr, *carved = nullptr;
    float *tables = nullptr;  // n_ang angle centres, n_u lateral centres, nz heights
    int *slice_bin = nullptr;
    int phase = 0;  // 0 statistics, 1 cuts, 2 finalised
};

namespace {

#define HB_CUDA(call)                              \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) {                   \
            hd::note_cuda_error(e_, #call);        \
            return HD_ERR_CUDA;                    \
        }                                          \
    } while (0)

struct BinDevice {
    int prev = -1;
    bool ok = true;
    explicit BinDevice(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~BinDevice()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

long long fixed_of(float v, double scale) { return llrint(static_cast<double>(v) * scale); }

hd_status make_binq(const hd_binned_params *p, hd::BinQ &b)
{
    auto finite = [](float v) { return std::isfinite(v); };
    if (!finite(p->angle_bin_deg) || !finite(p->u_bin_mm) || !finite(p->v_bin_mm) ||
        !finite(p->u_lo_mm) || !finite(p->v_lo_mm) || !finite(p->miss_wepl_mm))
        return HD_ERR_ARG;
    if (!(p->angle_bin_deg >= 1.0f / 16.0f && p->angle_bin_deg <= 360.0f)) return HD_ERR_RANGE;
    if (!(p->u_bin_mm >= 1.0f / 16.0f && p->u_bin_mm <= 4096.0f)) return HD_ERR_RANGE;
    if (!(p->v_bin_mm >= 1.0f / 16.0f && p->v_bin_mm <= 4096.0f)) return HD_ERR_RANGE;
    if (std::fabs(p->u_lo_mm) > 4096.0f || std::fabs(p->v_lo_mm) > 4096.0f) return HD_ERR_RANGE;
    if (std::fabs(p->miss_wepl_mm) >= 1024.0f) return HD_ERR_RANGE;
    if (p->n_u < 1 || p->n_v < 1 || p->k_sigma < 1 || p->k_sigma > 64) return HD_ERR_RANGE;
    if (p->window < 1 || p->window > 15 || p->window % 2 == 0) return HD_ERR_RANGE;
    if (p->min_count < 0 || p->min_count > p->window * p->window) return HD_ERR_RANGE;
    b.ang_q = fixed_of(p->angle_bin_deg, 65536.0);
    if (hd::kFull % b.ang_q != 0) return HD_ERR_RANGE;
    b.n_ang = static_cast<int>(hd::kFull / b.ang_q);
    b.n_u = p->n_u;
    b.n_v = p->n_v;
    if (static_cast<int64_t>(b.n_ang) * b.n_u * b.n_v > (int64_t(1) << 24)) return HD_ERR_RANGE;
    b.u_q = fixed_of(p->u_bin_mm, 65536.0);
    b.v_q = fixed_of(p->v_bin_mm, 65536.0);
    b.u_lo_q = fixed_of(p->u_lo_mm, 65536.0);
    b.v_lo_q = fixed_of(p->v_lo_mm, 65536.0);
    b.k = p->k_sigma;
    b.miss_q8 = fixed_of(p->miss_wepl_mm, 256.0);
    b.w = p->window;
    b.min_count = p->min_count;
    return HD_OK;
}

long long floordiv_host(long long a, long long b)  // b > 0
{
    long long q = a / b;
    if (a % b != 0 && a < 0) --q;
    return q;
}

void free_binned(hd_binned *b)
{
    if (!b) return;
    if (b->acc) cudaFree(b->acc);
    if (b->ctr) cudaFree(b->ctr);
    if (b->bits) cudaFree(b->bits);
    if (b->mask) cudaFree(b->mask);
    if (b->carved) cudaFree(b->carved);
    if (b->tables) cudaFree(b->tables);
    if (b->slice_bin) cudaFree(b->slice_bin);
    delete b;
}

// Every input pointer must be readable by the device.
hd_status check_inputs(const float *const *p, int k)
{
    for (int i = 0; i < k; ++i) {
        if (!p[i]) return HD_ERR_ARG;
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, p[i]) != cudaSuccess) {
            cudaGetLastError();
            return HD_ERR_ARG;
        }
        if (at.type == cudaMemoryTypeUnregistered) return HD_ERR_ARG;
    }
    return HD_OK;
}

hd_status pass(hd_binned *b, const float *angle_deg, const float *u_in, const float *v_in,
               const float *u_out, const float *v_out, const float *wepl, int64_t n, bool cut,
               cudaStream_t st)
{
    if (n < 0) return HD_ERR_ARG;
    if (n == 0) return HD_OK;
    const float *p[6] = {angle_deg, u_in, v_in, u_out, v_out, wepl};
    const hd_status v = check_inputs(p, 6);
    if (v != HD_OK) return v;
    const hd::Inputs in{angle_deg, u_in, v_in, u_out, v_out, wepl};
    const int grid = hd::grid_for(n, b->sm_count, hd::kPassBlocksPerSm);  // one wave
    if (cut)
        hd::binned_cut_kernel<<<grid, hd::kBinThreads, 0, st>>>(in, n, b->bq, b->acc, b->ctr);
    else
        hd::binned_stats_kernel<<<grid, hd::kBinThreads, 0, st>>>(in, n, b->bq, b->acc, b->ctr);
    HB_CUDA(cudaGetLastError());
    return HD_OK;
}

}  // namespace

extern "C" {

hd_status hd_binned_params_default(const hd_geometry *geom, hd_binned_params *out)
{
    if (!geom || !out) return HD_ERR_ARG;
    const hd_status gs = hd::check_geometry(geom);
    if (gs != HD_OK) return gs;
    out->angle_bin_deg = 4.0f;
    out->u_bin_mm = 1.0f;
    out->v_bin_mm = 5.0f;
    const double wx = static_cast<double>(geom->nx) * geom->sx;
    const double wy = static_cast<double>(geom->ny) * geom->sy;
    const double half_u = std::ceil(std::hypot(wx, wy) / 2.0 / out->u_bin_mm) * out->u_bin_mm;
    const double half_v =
        std::ceil(static_cast<double>(geom->nz) * geom->sz / 2.0 / out->v_bin_mm) * out->v_bin_mm;
    out->u_lo_mm = static_cast<float>(-half_u);
    out->v_lo_mm = static_cast<float>(-half_v);
    out->n_u = static_cast<int32_t>(std::lround(2.0 * half_u / out->u_bin_mm));
    out->n_v = static_cast<int32_t>(std::lround(2.0 * half_v / out->v_bin_mm));
    out->k_sigma = 3;
    out->miss_wepl_mm = 1.0f;
    out->window = 5;
    out->min_count = 11;
    return HD_OK;
}

hd_status hd_binned_create(const hd_geometry *geom, const hd_binned_params *params,
                           hd_binned **out)
{
    if (!out || !geom || !params) return HD_ERR_ARG;
    *out = nullptr;
    const hd_status gs = hd::check_geometry(geom);
    if (gs != HD_OK) return gs;
    hd::BinQ bq{};
    const hd_status ps = make_binq(params, bq);
    if (ps != HD_OK) return ps;
    hd_binned *b = new (std::nothrow) hd_binned();
    if (!b) return HD_ERR_NOMEM;
    b->geom = *geom;
    b->params = *params;
    b->bq = bq;
    if (!hd::make_cordic_table(b->cordic)) {
        delete b;
        return HD_ERR_RANGE;
    }
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) {
        hd::note_cuda_error(e, "hd_binned_create: device query");
        delete b;
        return HD_ERR_CUDA;
    }
    b->gq = hd::make_geomq(geom->nx, geom->ny, geom->nz, geom->sx, geom->sy, geom->sz,
                           geom->tracker_half_sep_mm);
    b->V = int64_t(geom->nx) * geom->ny * geom->nz;
    b->nb = int64_t(bq.n_ang) * bq.n_u * bq.n_v;
    const int64_t plane = int64_t(geom->nx) * geom->ny;
    b->wps = static_cast<int>((plane + 31) / 32);
    // line tables, computed as the method states them: centre angle ia
    // times the bin size, lateral centre lo + (iu + 1/2) size, slice centre
    // height from the Q16 slice thickness and its vertical bin
    const int nz = geom->nz;
    const size_t nt = static_cast<size_t>(bq.n_ang) + bq.n_u + nz;
    float *tab = new (std::nothrow) float[nt];
    int *sb = new (std::nothrow) int[nz];
    if (!tab || !sb) {
        delete[] tab;
        delete[] sb;
        delete b;
        return HD_ERR_NOMEM;
    }
    for (int ia = 0; ia < bq.n_ang; ++ia)
        tab[ia] = static_cast<float>(static_cast<double>(ia * bq.ang_q) / 65536.0);
    for (int iu = 0; iu < bq.n_u; ++iu)
        tab[bq.n_ang + iu] = static_cast<float>(
            static_cast<double>(2 * bq.u_lo_q + (2LL * iu + 1) * bq.u_q) / (2.0 * 65536.0));
    for (int z = 0; z < nz; ++z) {
        const long long c2 = (2LL * z + 1 - nz) * b->gq.sz;
        tab[bq.n_ang + bq.n_u + z] = static_cast<float>(static_cast<double>(c2) / (2.0 * 65536.0));
        const long long iv = floordiv_host(c2 - 2 * bq.v_lo_q, 2 * bq.v_q);
        sb[z] = (iv >= 0 && iv < bq.n_v) ? static_cast<int>(iv) : -1;
    }
    bool ok = true;
    auto alloc = [&](void **p, size_t bytes) {
        if (!ok) return;
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            ok = false;
        }
    };
    alloc(reinterpret_cast<void **>(&b->acc), sizeof(unsigned long long) * hd::kAccWords * b->nb);
    alloc(reinterpret_cast<void **>(&b->ctr), sizeof(unsigned long long) * hd::kCtrWords);
    alloc(reinterpret_cast<void **>(&b->bits), sizeof(uint32_t) * size_t(b->wps) * nz);
    alloc(reinterpret_cast<void **>(&b->mask), size_t(b->V));
    alloc(reinterpret_cast<void **>(&b->carved), size_t(b->V));
    alloc(reinterpret_cast<void **>(&b->tables), sizeof(float) * nt);
    alloc(reinterpret_cast<void **>(&b->slice_bin), sizeof(int) * nz);
    if (ok) {
        cudaError_t c = cudaMemcpy(b->tables, tab, sizeof(float) * nt, cudaMemcpyHostToDevice);
        if (c == cudaSuccess)
            c = cudaMemcpy(b->slice_bin, sb, sizeof(int) * nz, cudaMemcpyHostToDevice);
        if (c == cudaSuccess)
            c = cudaMemset(b->acc, 0, sizeof(unsigned long long) * hd::kAccWords * b->nb);
        if (c == cudaSuccess) c = cudaMemset(b->ctr, 0, sizeof(unsigned long long) * hd::kCtrWords);
        if (c == cudaSuccess) c = cudaDeviceSynchronize();
        if (c != cudaSuccess) {
            hd::note_cuda_error(c, "hd_binned_create: initialise");
            delete[] tab;
            delete[] sb;
            free_binned(b);
            return HD_ERR_CUDA;
        }
    }
    delete[] tab;
    delete[] sb;
    if (!ok) {
        free_binned(b);
        return HD_ERR_NOMEM;
    }
    // the largest slice bitmap any object uses, so objects of different
    // sizes never lower one another's limit
    if (cudaFuncSetAttribute(hd::binned_carve_kernel<true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sizeof(uint32_t) * hd::kMaxSmemWords)) !=
        cudaSuccess) {
        cudaGetLastError();
        free_binned(b);
        return HD_ERR_CUDA;
    }
    *out = b;
    return HD_OK;
}

hd_status hd_binned_destroy(hd_binned *b)
{
    if (!b) return HD_ERR_ARG;
    BinDevice g(b->device);
    cudaDeviceSynchronize();
    free_binned(b);
    return HD_OK;
}

hd_status hd_binned_reset(hd_binned *b, void *stream)
{
    if (!b) return HD_ERR_ARG;
    BinDevice g(b->device);
    if (!g.ok) return HD_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    HB_CUDA(cudaMemsetAsync(b->acc, 0, sizeof(unsigned long long) * hd::kAccWords * b->nb, st));
    HB_CUDA(cudaMemsetAsync(b->ctr, 0, sizeof(unsigned long long) * hd::kCtrWords, st));
    b->phase = 0;
    return HD_OK;
}

hd_status hd_binned_add_histories(hd_binned *b, const float *angle_deg, const float *u_in,
                                  const float *v_in, const float *u_out, const float *v_out,
                                  const float *wepl, int64_t n, void *stream)
{
    if (!b) return HD_ERR_ARG;
    if (b->phase != 0) return HD_ERR_STATE;
    BinDevice g(b->device);
    if (!g.ok) return HD_ERR_CUDA;
    return pass(b, angle_deg, u_in, v_in, u_out, v_out, wepl, n, false,
                static_cast<cudaStream_t>(stream));
}

hd_status hd_binned_cut_histories(hd_binned *b, const float *angle_deg, const float *u_in,
                                  const float *v_in, const float *u_out, const float *v_out,
                                  const float *wepl, int64_t n, void *stream)
{
    if (!b) return HD_ERR_ARG;
    if (b->phase == 2) return HD_ERR_STATE;
    BinDevice g(b->device);
    if (!g.ok) return HD_ERR_CUDA;
    const hd_status s = pass(b, angle_deg, u_in, v_in, u_out, v_out, wepl, n, true,
                             static_cast<cudaStream_t>(stream));
    if (s == HD_OK) b->phase = 1;
    return s;
}

hd_status hd_binned_finalize(hd_binned *b, void *stream)
{
    if (!b) return HD_ERR_ARG;
    if (b->phase == 0) return HD_ERR_STATE;
    BinDevice g(b->device);
    if (!g.ok) return HD_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nz = b->geom.nz;
    HB_CUDA(cudaMemsetAsync(b->ctr + 2, 0, sizeof(unsigned long long) * 4, st));
    HB_CUDA(cudaMemsetAsync(b->bits, 0xff, sizeof(uint32_t) * size_t(b->wps) * nz, st));
    hd::binned_bins_kernel<<<hd::grid_for(b->nb, b->sm_count), hd::kBinThreads, 0, st>>>(
        b->acc, b->nb, b->bq.miss_q8, b->ctr);
    HB_CUDA(cudaGetLastError());
    const hd::LineTables t{b->tables, b->tables + b->bq.n_ang, b->tables + b->bq.n_ang + b->bq.n_u,
                           b->slice_bin};
    const dim3 cg(static_cast<unsigned>(b->bq.n_ang), static_cast<unsigned>(nz));
    if (b->wps <= hd::kMaxSmemWords)
        hd::binned_carve_kernel<true><<<cg, hd::kCarveThreads, sizeof(uint32_t) * b->wps, st>>>(
            b->acc, b->bq, b->gq, b->cordic, t, b->bits, b->wps, b->ctr);
    else
        hd::binned_carve_kernel<false><<<cg, hd::kCarveThreads, 0, st>>>(
            b->acc, b->bq, b->gq, b->cordic, t, b->bits, b->wps, b->ctr);
    HB_CUDA(cudaGetLastError());
    const dim3 fb(32, 8);
    const dim3 fg(static_cast<unsigned>((b->geom.nx + 31) / 32),
                  static_cast<unsigned>((b->geom.ny + 7) / 8), static_cast<unsigned>(nz));
    hd::binned_filter_kernel<<<fg, fb, 0, st>>>(b->bits, b->wps, b->geom.nx, b->geom.ny,
                                                 b->bq.w / 2, b->bq.min_count, b->mask, b->carved);
    HB_CUDA(cudaGetLastError());
    b->phase = 2;
    return HD_OK;
}

hd_status hd_binned_run(hd_binned *b, const float *angle_deg, const float *u_in,
                        const float *v_in, const float *u_out, const float *v_out,
                        const float *wepl, int64_t n, void *stream)
{
    hd_status s = hd_binned_reset(b, stream);
    if (s == HD_OK) s = hd_binned_add_histories(b, angle_deg, u_in, v_in, u_out, v_out, wepl, n, stream);
    if (s == HD_OK) s = hd_binned_cut_histories(b, angle_deg, u_in, v_in, u_out, v_out, wepl, n, stream);
    if (s == HD_OK && b->phase == 0) b->phase = 1;  // n == 0: nothing to cut
    if (s == HD_OK) s = hd_binned_finalize(b, stream);
    return s;
}

hd_status hd_binned_get_image(hd_binned *b, int32_t which, uint8_t *dst, int64_t n,
                              int32_t dst_on_device, void *stream)
{
    if (!b || !dst || (which != HD_BINNED_HULL && which != HD_BINNED_CARVED)) return HD_ERR_ARG;
    if (n < b->V) return HD_ERR_ARG;
    if (b->phase != 2) return HD_ERR_STATE;
    BinDevice g(b->device);
    if (!g.ok) return HD_ERR_CUDA;
    HB_CUDA(cudaMemcpyAsync(dst, which == HD_BINNED_HULL ? b->mask : b->carved, size_t(b->V),
                            dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            static_cast<cudaStream_t>(stream)));
    return HD_OK;
}

hd_status hd_binned_get_bins(hd_binned *b, int64_t *dst, int64_t n_bins, int32_t dst_on_device,
                             void *stream)
{
    if (!b || !dst || n_bins < b->nb) return HD_ERR_ARG;
    BinDevice g(b->device);
    if (!g.ok) return HD_ERR_CUDA;
    HB_CUDA(cudaMemcpyAsync(dst, b->acc, sizeof(int64_t) * hd::kAccWords * b->nb,
                            dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            static_cast<cudaStream_t>(stream)));
    return HD_OK;
}

hd_status hd_binned_get_stats(hd_binned *b, hd_binned_stats *out, void *stream)
{
    if (!b || !out) return HD_ERR_ARG;
    BinDevice g(b->device);
    if (!g.ok) return HD_ERR_CUDA;
    unsigned long long c[hd::kCtrWords];
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    HB_CUDA(cudaMemcpyAsync(c, b->ctr, sizeof(c), cudaMemcpyDeviceToHost, st));
    HB_CUDA(cudaStreamSynchronize(st));
    out->histories_binned = static_cast<int64_t>(c[0]);
    out->histories_cut = static_cast<int64_t>(c[1]);
    out->bins = b->nb;
    out->bins_used = static_cast<int64_t>(c[2]);
    out->bins_missed = static_cast<int64_t>(c[3]);
    out->lines = static_cast<int64_t>(c[4]);
    out->lines_outside = static_cast<int64_t>(c[5]);
    return HD_OK;
}

}  // extern "C"
