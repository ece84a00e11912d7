// Per-voxel decisions from the resident counts, and mask packing/compaction.
//
//   H_1 = V \ U A_i = {v : N(v) = 0}                       (Eq. 3.3, Alg. 1)
//   H_2 = {v : max_{w in B(v)} N(v) - N(w) < N_t}           (Eq. 3.6, Alg. 2)
//   M_t = M(v*), v* the last voxel (x-fastest order) with the steepest drop
//         max_{w in B(v)} M(v) - M(w) of its slice; H_3 = {v : M(v) >= M_t}
//         (Eq. 3.10, Alg. 3, per slice as Sec. 3.4 describes; ">" by flag)
// B(v) = {w : d(v, w) <= 1} (Eq. 3.5) in voxel-index units: v and its face
// neighbours inside the grid (6), or the in-plane ones (4).  Slices with no
// drop (maximum 0) have no edge and get H_3 = 0.
#include "hd_internal.cuh"

namespace hd {

namespace {

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
        v = t > v ? t : v;
    }
    return v;
}

// Steepest drop per slice (or over the volume): max of the packed key
// (S(v) << 32) | index, so the largest S wins and, among equal S, the
// largest index, which is what the ">=" update of Alg. 3 leaves behind.
__global__ void __launch_bounds__(256) sm_slope_kernel(const uint32_t *__restrict__ M, int nx,
                                                       int ny, int nz, int per_slice, int nbhd,
                                                       unsigned long long *slice_key)
{
    const int z = blockIdx.y;
    const int plane = nx * ny;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long key = 0;
    bool have = false;
    if (q < plane) {
        const int x = q % nx, y = q / nx;
        const int64_t v = static_cast<int64_t>(z) * plane + q;
        const uint32_t m = M[v];
        uint32_t mn = m;
        if (x > 0) mn = min(mn, M[v - 1]);
        if (x + 1 < nx) mn = min(mn, M[v + 1]);
        if (y > 0) mn = min(mn, M[v - nx]);
        if (y + 1 < ny) mn = min(mn, M[v + nx]);
        if (!per_slice && nbhd == 6) {
            if (z > 0) mn = min(mn, M[v - plane]);
            if (z + 1 < nz) mn = min(mn, M[v + plane]);
        }
        const unsigned long long S = m - mn;
        const unsigned long long id = per_slice ? static_cast<unsigned long long>(q)
                                                : static_cast<unsigned long long>(v);
        key = (S << 32) | id;
        have = true;
    }
    // a lane without a voxel contributes 0, the value the keys start from,
    // so it changes no maximum; the block's maximum goes out in one atomic
    // (one per warp made the same-address atomics of a slice the bottleneck)
    __shared__ unsigned long long s_max[8];
    key = warp_max_u64(have ? key : 0ull);
    if ((threadIdx.x & 31u) == 0) s_max[threadIdx.x >> 5] = key;
    __syncthreads();
    if (threadIdx.x < 32) {
        key = threadIdx.x < (blockDim.x >> 5) ? s_max[threadIdx.x] : 0ull;
        key = warp_max_u64(key);
        if (threadIdx.x == 0 && key != 0) atomicMax(&slice_key[per_slice ? z : 0], key);
    }
}

__global__ void sm_threshold_kernel(const uint32_t *__restrict__ M, int nx, int ny, int nz,
                                    int per_slice, const unsigned long long *slice_key,
                                    uint32_t *mt, uint32_t *slope, long long *index)
{
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= nz) return;
    const unsigned long long key = slice_key[per_slice ? z : 0];
    const long long plane = static_cast<long long>(nx) * ny;
    const long long id = static_cast<long long>(key & 0xffffffffull);
    const long long v = per_slice ? z * plane + id : id;
    slope[z] = static_cast<uint32_t>(key >> 32);
    index[z] = v;
    mt[z] = M[v];
}

__global__ void __launch_bounds__(256) decide_kernel(DecideArgs a)
{
    const int z = blockIdx.y;
    const int plane = a.nx * a.ny;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= plane) return;
    const int x = q % a.nx, y = q / a.nx;
    const int64_t v = static_cast<int64_t>(z) * plane + q;
    if (a.methods & HD_SC) a.H1[v] = a.N[v] == 0;  // Eq. 3.3
    if (a.methods & HD_MSC) {
        const uint32_t n = a.N[v];
        uint32_t mn = n;
        if (x > 0) mn = min(mn, a.N[v - 1]);
        if (x + 1 < a.nx) mn = min(mn, a.N[v + 1]);
        if (y > 0) mn = min(mn, a.N[v - a.nx]);
        if (y + 1 < a.ny) mn = min(mn, a.N[v + a.nx]);
        if (a.nbhd == 6) {
            if (z > 0) mn = min(mn, a.N[v - plane]);
            if (z + 1 < a.nz) mn = min(mn, a.N[v + plane]);
        }
        a.H2[v] = (static_cast<long long>(n) - static_cast<long long>(mn)) <
                  static_cast<long long>(a.nt);
    }
    if (a.methods & HD_SM) {
        const uint32_t m = a.M[v];
        const uint32_t t = a.mt[z];
        const bool edge = a.slope[z] != 0;
        a.H3[v] = edge && (a.sm_ge ? (m >= t) : (m > t));
    }
}

__global__ void pack_bits_kernel(const uint8_t *__restrict__ mask, int64_t V, uint32_t *bits)
{
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t words = (V + 31) / 32;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
         i < words * 32; i += stride) {
        const bool b = i < V && mask[i] != 0;
        const unsigned w = __ballot_sync(0xffffffffu, b);
        if ((threadIdx.x & 31u) == 0) bits[i >> 5] = w;
    }
}

constexpr int kCompactBlock = 1024;

__global__ void __launch_bounds__(kCompactBlock) compact_count_kernel(const uint8_t *mask,
                                                                      int64_t V,
                                                                      uint32_t *block_counts)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kCompactBlock + threadIdx.x;
    const int c = __syncthreads_count(i < V && mask[i] != 0);
    if (threadIdx.x == 0) block_counts[blockIdx.x] = static_cast<uint32_t>(c);
}

// Exclusive scan of block counts in one block; writes the total.
__global__ void __launch_bounds__(1024) compact_scan_kernel(uint32_t *block_counts, int64_t nb,
                                                            unsigned long long *d_total)
{
    __shared__ unsigned long long warp_sums[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    for (int64_t base = 0; base < nb; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const unsigned long long v = i < nb ? block_counts[i] : 0ull;
        unsigned long long incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= static_cast<unsigned>(o)) incl += t;
        }
        if (lane == 31) warp_sums[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            unsigned long long ws = warp_sums[lane];
            unsigned long long wincl = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long t = __shfl_up_sync(0xffffffffu, wincl, o);
                if (lane >= static_cast<unsigned>(o)) wincl += t;
            }
            warp_sums[lane] = wincl - ws;  // exclusive warp offsets
        }
        __syncthreads();
        const unsigned long long excl = carry + warp_sums[wid] + incl - v;
        if (i < nb) block_counts[i] = static_cast<uint32_t>(excl);
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *d_total = carry;
}

__global__ void __launch_bounds__(kCompactBlock) compact_write_kernel(const uint8_t *mask,
                                                                      int64_t V,
                                                                      const uint32_t *offsets,
                                                                      int32_t *out,
                                                                      int64_t capacity)
{
    __shared__ unsigned warp_off[kCompactBlock / 32];
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kCompactBlock + threadIdx.x;
    const bool b = i < V && mask[i] != 0;
    const unsigned bal = __ballot_sync(0xffffffffu, b);
    const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    if (lane == 0) warp_off[wid] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        for (int w = 0; w < kCompactBlock / 32; ++w) {
            const unsigned c = warp_off[w];
            warp_off[w] = acc;
            acc += c;
        }
    }
    __syncthreads();
    if (b) {
        const int64_t pos = static_cast<int64_t>(offsets[blockIdx.x]) + warp_off[wid] +
                            __popc(bal & ((1u << lane) - 1u));
        if (pos < capacity) out[pos] = static_cast<int32_t>(i);
    }
}

// Sums of the two count volumes (64-bit, exact): grid-stride, four words
// per thread and step, a warp reduction and one atomic per warp and volume.
__global__ void __launch_bounds__(256) volume_sums_kernel(const uint32_t *__restrict__ N,
                                                          const uint32_t *__restrict__ M,
                                                          int64_t V, unsigned long long *out)
{
    unsigned long long sn = 0, sm = 0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < V;
         i += stride) {
        if (N) sn += N[i];
        if (M) sm += M[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sn += __shfl_xor_sync(0xffffffffu, sn, o);
        sm += __shfl_xor_sync(0xffffffffu, sm, o);
    }
    if ((threadIdx.x & 31u) == 0) {
        if (sn) atomicAdd(&out[0], sn);
        if (sm) atomicAdd(&out[1], sm);
    }
}

}  // namespace

cudaError_t launch_volume_sums(const uint32_t *N, const uint32_t *M, int64_t V,
                               unsigned long long *out, int sm_count, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess || V <= 0 || (!N && !M)) return e;
    int64_t blocks = (V + 255) / 256;
    const int64_t cap = static_cast<int64_t>(sm_count > 0 ? sm_count : 1) * 4;
    if (blocks > cap) blocks = cap;
    volume_sums_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(N, M, V, out);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const DecideArgs &a, int sm_count, cudaStream_t s)
{
    (void)sm_count;
    const int plane = a.nx * a.ny;
    const dim3 grid((plane + 255) / 256, a.nz);
    if (a.methods & HD_SM) {
        cudaError_t e = cudaMemsetAsync(a.slice_key, 0, sizeof(unsigned long long) * a.nz, s);
        if (e != cudaSuccess) return e;
        sm_slope_kernel<<<grid, 256, 0, s>>>(a.M, a.nx, a.ny, a.nz, a.sm_per_slice, a.nbhd,
                                             a.slice_key);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        sm_threshold_kernel<<<(a.nz + 127) / 128, 128, 0, s>>>(a.M, a.nx, a.ny, a.nz,
                                                               a.sm_per_slice, a.slice_key, a.mt,
                                                               a.slope, a.index);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    decide_kernel<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pack_bits(const uint8_t *mask, int64_t V, uint32_t *bits, cudaStream_t s)
{
    const int64_t threads = ((V + 31) / 32) * 32;
    int64_t blocks = (threads + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    pack_bits_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(mask, V, bits);
    return cudaGetLastError();
}

cudaError_t launch_compact(const uint8_t *mask, int64_t V, int32_t *out, int64_t capacity,
                           uint32_t *block_counts, unsigned long long *d_count, cudaStream_t s)
{
    const int64_t nb = (V + kCompactBlock - 1) / kCompactBlock;
    compact_count_kernel<<<static_cast<unsigned>(nb), kCompactBlock, 0, s>>>(mask, V,
                                                                            block_counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    compact_scan_kernel<<<1, 1024, 0, s>>>(block_counts, nb, d_count);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    compact_write_kernel<<<static_cast<unsigned>(nb), kCompactBlock, 0, s>>>(
        mask, V, block_counts, out, capacity);
    return cudaGetLastError();
}

}  // namespace hd
