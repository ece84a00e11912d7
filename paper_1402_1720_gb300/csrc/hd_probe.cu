// Atomic-throughput probe: the ceilings a traversal that spent one atomic per
// voxel-step could reach on this GPU, measured with plain kernels that do
// nothing else (a measurement aid for the roofline; the paper has no
// counterpart).  Addresses come from a per-thread xorshift generator
// (Marsaglia 2003) masked into a power-of-two buffer, so every access stays
// in bounds; every loop has a fixed trip count.
#include <cuda_runtime.h>

#include "hd_internal.cuh"

namespace {

constexpr int kProbeThreads = 1024;
constexpr int kSmemWords = 1 << 15;  // 128 KB, about one config-2 tile
constexpr int kSmemIters = 2048;     // atomics per thread
constexpr int kGlobalIters = 256;

__device__ __forceinline__ unsigned xorshift32(unsigned &x)
{
    x ^= x << 13;
    x ^= x >> 17;
    x ^= x << 5;
    return x;
}

// kRandom: uniformly random words; otherwise lane l of a warp hits word
// (32 w + l + 1024 k) mod size, so a warp touches 32 consecutive words.
template <bool kRandom>
__global__ void __launch_bounds__(kProbeThreads) probe_smem_kernel(unsigned *sink)
{
    extern __shared__ unsigned sm[];
    for (int i = threadIdx.x; i < kSmemWords; i += blockDim.x) sm[i] = 0;
    __syncthreads();
    unsigned x = 0x9e3779b9u * (blockIdx.x * blockDim.x + threadIdx.x + 1u);
    for (int k = 0; k < kSmemIters; ++k) {
        const unsigned idx = kRandom ? (xorshift32(x) & (kSmemWords - 1))
                                     : ((threadIdx.x + (static_cast<unsigned>(k) << 10)) &
                                        (kSmemWords - 1));
        atomicAdd(&sm[idx], 1u);
    }
    __syncthreads();
    unsigned acc = 0;
    for (int i = threadIdx.x; i < kSmemWords; i += blockDim.x) acc += sm[i];
    if (acc == 0xffffffffu) atomicAdd(sink, 1u);  // keeps the work observable
}

__global__ void __launch_bounds__(kProbeThreads) probe_global_kernel(unsigned *buf, unsigned mask)
{
    unsigned x = 0x85ebca6bu * (blockIdx.x * blockDim.x + threadIdx.x + 1u);
    for (int k = 0; k < kGlobalIters; ++k) atomicAdd(&buf[xorshift32(x) & mask], 1u);
}

}  // namespace

extern "C" {

hd_status hd_probe_atomics(int32_t kind, double *ops_per_s)
{
    if (!ops_per_s || kind < HD_PROBE_SMEM_RANDOM || kind > HD_PROBE_HBM_RANDOM) return HD_ERR_ARG;
    *ops_per_s = 0.0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    const bool smem = kind == HD_PROBE_SMEM_RANDOM || kind == HD_PROBE_SMEM_COHERENT;
    // global buffers: 16 MB stays in L2, 2 GB does not
    const size_t words = smem ? 1 : (kind == HD_PROBE_L2_RANDOM ? (size_t(1) << 22) : (size_t(1) << 29));
    unsigned *buf = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    hd_status r = HD_OK;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && r == HD_OK) {
            cudaGetLastError();
            r = (e == cudaErrorMemoryAllocation) ? HD_ERR_NOMEM : HD_ERR_CUDA;
        }
        return r == HD_OK;
    };
    if (ok(cudaMalloc(&buf, sizeof(unsigned) * words)) &&
        ok(cudaMemset(buf, 0, sizeof(unsigned) * words)) &&
        ok(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) && ok(cudaEventCreate(&e0)) &&
        ok(cudaEventCreate(&e1))) {
        const size_t smem_bytes = sizeof(unsigned) * kSmemWords;
        if (smem) {
            ok(cudaFuncSetAttribute(probe_smem_kernel<true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(smem_bytes)));
            ok(cudaFuncSetAttribute(probe_smem_kernel<false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(smem_bytes)));
        }
        const int grid = smem ? sms : 2 * sms;
        const double ops = static_cast<double>(grid) * kProbeThreads *
                           (smem ? kSmemIters : kGlobalIters);
        float best = 0.0f;
        for (int rep = 0; rep < 4 && r == HD_OK; ++rep) {  // the first is a warm-up
            ok(cudaEventRecord(e0, st));
            if (kind == HD_PROBE_SMEM_RANDOM)
                probe_smem_kernel<true><<<grid, kProbeThreads, smem_bytes, st>>>(buf);
            else if (kind == HD_PROBE_SMEM_COHERENT)
                probe_smem_kernel<false><<<grid, kProbeThreads, smem_bytes, st>>>(buf);
            else
                probe_global_kernel<<<grid, kProbeThreads, 0, st>>>(
                    buf, static_cast<unsigned>(words - 1));
            ok(cudaGetLastError());
            ok(cudaEventRecord(e1, st));
            ok(cudaEventSynchronize(e1));
            float ms = 0.0f;
            if (r == HD_OK && ok(cudaEventElapsedTime(&ms, e0, e1)) && rep > 0 && ms > 0.0f &&
                (best == 0.0f || ms < best))
                best = ms;
        }
        if (r == HD_OK && best > 0.0f) *ops_per_s = ops / (best * 1e-3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (buf) cudaFree(buf);
    return r;
}

}  // extern "C"
