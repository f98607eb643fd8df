// noalloc.cu -- dense rotation for callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc: a plug-in running inside
// a host program whose device memory is already fully reserved by that
// program's own pool allocator, code running under a fixed per-client memory
// limit (for instance an MPS client), or a latency-critical loop where a
// cudaMalloc/cudaFree would synchronise the whole device.  For them this file
// provides dmrg_rotate_ops_noalloc(): the same dense rotation as
// dmrg_rotate_ops(), but with no handle and no caller workspace.  Its scratch
// (packed operands, the intermediate product and the device status word) is a
// file-scope static __device__ array of fixed size, so every GPU that loads
// the library holds these bytes until the process exits.
//
// Host code cannot use the array's name as a device address (it is a host-side
// stand-in).  The first call on each device, with that device current, asks
// the runtime for the real address with cudaGetSymbolAddress and keeps it; that
// first call should therefore come before any stream capture.  Every call
// shares the one array: calls whose work overlaps on the GPU (different
// streams, different host threads) race on it and must be serialised by the
// caller.  Nothing in the array needs to start at zero: every scratch element
// the kernels read was written earlier in the same call.
#include <cuda_runtime.h>

#include <mutex>

#include "api_common.h"

namespace {

constexpr size_t kStatusBytes = 256;                        // status word + reduction scratch
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB of workspace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kStatusBytes + kNoAllocScratchBytes];

struct NoAllocDevice {
    bool ready = false;
    dmrg_handle_s h;             // host-side bookkeeping only; owns no device memory
    unsigned char* ws = nullptr;  // device address of the workspace part of the array
};

constexpr int kMaxDevices = 64;
NoAllocDevice g_devices[kMaxDevices];
std::mutex g_setup_mutex;

dmrg_status setup_device(int dev, NoAllocDevice*& out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    NoAllocDevice& c = g_devices[dev];
    if (!c.ready) {
        void* base = nullptr;
        if (cudaGetSymbolAddress(&base, g_noalloc_scratch) != cudaSuccess || base == nullptr)
            return DMRG_ERR_CUDA;
        dmrg_handle_s& h = c.h;
        h.device = dev;
        if (cudaDeviceGetAttribute(&h.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&h.cc_major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&h.cc_minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
            return DMRG_ERR_CUDA;
        h.d_status = static_cast<unsigned*>(base);
        h.d_scratch = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + 64);
        c.ws = static_cast<unsigned char*>(base) + kStatusBytes;
        c.ready = true;
    }
    out = &c;
    return DMRG_OK;
}

}  // namespace

extern "C" DMRG_API dmrg_status dmrg_rotate_ops_noalloc(const double* U, int64_t m, int d,
                                                        int64_t mp, const void* O, int in_is_fp64,
                                                        int64_t K, void* Oout,
                                                        dmrg_precision precision,
                                                        dmrg_stream_t stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DMRG_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return DMRG_ERR_UNSUPPORTED;
    NoAllocDevice* c = nullptr;
    dmrg_status st = setup_device(dev, c);
    if (st != DMRG_OK) return st;
    dmrg_handle h = &c->h;
    st = dmrg::check_dense_args(h, K, m, d, mp, precision);
    if (st != DMRG_OK) return st;
    if (K == 0) return DMRG_OK;
    if (!U || !O || !Oout) return DMRG_ERR_INVALID_ARG;
    if (precision == DMRG_PREC_FP64 && !in_is_fp64) return DMRG_ERR_INVALID_ARG;
    const dmrg::DenseDims D = dmrg::dense_dims(K, m, d, mp, precision);
    if (D.ws.total > kNoAllocScratchBytes) return DMRG_ERR_WORKSPACE;  // problem too large
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (precision == DMRG_PREC_FP64 || precision == DMRG_PREC_FP32)
        return dmrg::dense_simt_forward(h, U, m, d, mp, O, in_is_fp64, K, Oout, precision, c->ws, s);
    if (!dmrg::tc_supported(h)) return DMRG_ERR_UNSUPPORTED;
    const dmrg::TcMode mode = (precision == DMRG_PREC_BF16X3) ? dmrg::TC_BF16X3 : dmrg::TC_TF32;
    dmrg::TcConfig cfg;
    cfg.tile_n_max = 256;
    cfg.row_bytes = 128;
    cfg.pair = 1;
    cfg.stages = dmrg::tc_stages_for(mode, cfg);
    return dmrg::dense_tc_forward(h, U, m, d, mp, O, in_is_fp64, K, Oout, precision, c->ws, cfg,
                                  cfg, s);
}
