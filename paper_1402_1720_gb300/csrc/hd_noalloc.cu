// Allocation-free accumulation of missed/hit path counts.
//
// Some callers cannot allocate device memory at the point where they want to
// run the traversal: code running inside a CUDA stream capture that must not
// grow the graph with allocation nodes, callers that hand out all device
// memory through their own pool and forbid cudaMalloc/cudaFree after start-up,
// and real-time paths that cannot afford the implicit synchronisation of an
// allocation.  This entry point serves them: it takes the caller's input and
// output buffers and keeps its only scratch (the compacted traversal records
// and their counters) in one fixed-size array that lives in the library's
// device image, so no call allocates anything.
//
// The array is shared by every call in the process on a given device and
// keeps what the last call left in it; each call clears the counters it
// needs before using them.  Calls that overlap on the GPU (on different
// streams, or from different host threads without ordering) race on it.
#include <cmath>
#include <mutex>

#include "hd_geom.cuh"

namespace {

// Histories per call (a multiple of 4); the records take 7 int32 each.
constexpr int64_t kNoAllocMaxHistories = int64_t(1) << 18;
static_assert(kNoAllocMaxHistories % 4 == 0, "record arrays are padded to four slots");
constexpr size_t kNoAllocCtrlBytes = 256;
constexpr size_t kNoAllocBytes =
    kNoAllocCtrlBytes + sizeof(int32_t) * 7 * static_cast<size_t>(kNoAllocMaxHistories);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];
static_assert(sizeof(hd::Ctrl) <= kNoAllocCtrlBytes, "the counters must fit their slot");

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

// Address of the scratch array on `dev` (the current device).  In host code
// the symbol itself is only a host-side stand-in, so the device address has
// to be asked for once per device; that first look-up may load the module
// and must not happen while `stream` is being captured (HD_ERR_STATE then).
// The address is cached for the life of the process: after a reset of the
// device (cudaDeviceReset) the module is loaded again and the array may
// move, so this entry point is not for use across a device reset.
hd_status scratch_for(int dev, cudaStream_t stream, void **addr, int *sm_count)
{
    if (dev < 0 || dev >= kMaxDevices) return HD_ERR_RANGE;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) {
            cudaGetLastError();
            return HD_ERR_CUDA;
        }
        if (cs != cudaStreamCaptureStatusNone) return HD_ERR_STATE;
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return HD_ERR_CUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return HD_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
        g_sm_count[dev] = sms;
    }
    *addr = g_scratch_addr[dev];
    *sm_count = g_sm_count[dev];
    return HD_OK;
}

// The gantry-rotation constants (the scans' table), built once per process.
bool cordic_constants(hd::Cordic &c)
{
    static std::once_flag once;
    static hd::Cordic table;
    static bool ok = false;
    std::call_once(once, [] { ok = hd::make_cordic_table(table); });
    c = table;
    return ok;
}

}  // namespace

extern "C" hd_status hd_accumulate_noalloc(const hd_geometry *geom, const hd_params *params,
                                           const float *angle_deg, const float *u_in,
                                           const float *v_in, const float *u_out,
                                           const float *v_out, const float *wepl, int64_t n,
                                           uint32_t *N, uint32_t *M, void *stream)
{
    if (!geom || !params || n < 0) return HD_ERR_ARG;
    if (n > kNoAllocMaxHistories) return HD_ERR_RANGE;
    const hd_status gs = hd::check_geometry(geom);
    if (gs != HD_OK) return gs;
    if (std::isnan(params->wepl_miss_lt) || std::isnan(params->wepl_hit_gt) ||
        params->wepl_miss_lt > params->wepl_hit_gt)
        return HD_ERR_ARG;
    const uint32_t m = params->methods;
    if (m == 0 || (m & ~uint32_t(HD_SC | HD_MSC | HD_SM))) return HD_ERR_ARG;
    const int use_miss = (m & (HD_SC | HD_MSC)) ? 1 : 0;
    const int use_hit = (m & HD_SM) ? 1 : 0;
    if ((use_miss && !N) || (use_hit && !M)) return HD_ERR_ARG;
    if (n == 0) return HD_OK;
    if (!angle_deg || !u_in || !v_in || !u_out || !v_out || !wepl) return HD_ERR_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    void *base = nullptr;
    int sm_count = 0;
    const hd_status st = scratch_for(dev, static_cast<cudaStream_t>(stream), &base, &sm_count);
    if (st != HD_OK) return st;
    hd::Cordic cordic;
    if (!cordic_constants(cordic)) return HD_ERR_RANGE;

    const hd::GeomQ gq = hd::make_geomq(geom->nx, geom->ny, geom->nz, geom->sx, geom->sy,
                                        geom->sz, geom->tracker_half_sep_mm);
    hd::TilePlan tp{};  // no tiles: every record takes the global-memory path
    tp.nx = geom->nx;
    tp.ny = geom->ny;
    tp.nz = geom->nz;
    tp.tx = geom->nx;
    tp.ty = geom->ny;
    tp.tz = geom->nz;
    tp.ntx = tp.nty = tp.ntz = 1;

    auto *bytes = static_cast<unsigned char *>(base);
    hd::Ctrl *ctrl = reinterpret_cast<hd::Ctrl *>(bytes);
    int32_t *rec_base = reinterpret_cast<int32_t *>(bytes + kNoAllocCtrlBytes);
    hd::Records rec;  // seven arrays of n slots, each on a 16-byte boundary
    const size_t stride = static_cast<size_t>(hd::records_stride(n));
    for (int a = 0; a < 6; ++a) rec.g[a] = rec_base + a * stride;
    rec.status = rec_base + 6 * stride;
    rec.glist = nullptr;  // the global pass finds its records by their status words
    rec.cap = n;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    hd::Inputs in{angle_deg, u_in, v_in, u_out, v_out, wepl};
    cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(hd::Ctrl), s);
    if (e == cudaSuccess)
        e = hd::launch_ingest(in, n, gq, cordic, params->wepl_miss_lt, params->wepl_hit_gt,
                              use_miss, use_hit, tp, rec, ctrl, nullptr, nullptr, nullptr, 0,
                              sm_count, s);
    if (e == cudaSuccess)
        e = hd::launch_trace_global(rec, ctrl, n, gq, use_miss ? N : nullptr,
                                    use_hit ? M : nullptr, 0, sm_count, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    return HD_OK;
}
