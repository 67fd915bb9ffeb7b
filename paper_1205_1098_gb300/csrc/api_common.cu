// Utility entry points: version, status strings, argument diagnostics,
// device facts and the device status word.
#include "internal.cuh"
#include <mutex>
#include <vector>

namespace bto {

static thread_local int g_invalid_arg = 0;
void set_invalid_arg(int pos) { g_invalid_arg = pos; }
void clear_invalid_arg() { g_invalid_arg = 0; }
int last_invalid_arg() { return g_invalid_arg; }

bool device_info(DeviceInfo* out) {
    static std::mutex mu;
    static std::vector<DeviceInfo> cache;
    static std::vector<bool> have;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= dev) { cache.resize(dev + 1); have.resize(dev + 1, false); }
    if (!have[dev]) {
        DeviceInfo d;
        if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return false;
        if (cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return false;
        int coop = 0;
        if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess)
            return false;
        d.coop = coop != 0;
        cache[dev] = d;
        have[dev] = true;
    }
    *out = cache[dev];
    return true;
}

}  // namespace bto

using namespace bto;

extern "C" int bto_version(void) { return 100; }

extern "C" const char* bto_status_string(int s) {
    switch (s) {
        case BTO_OK: return "BTO_OK: success";
        case BTO_ERR_INVALID_VALUE: return "BTO_ERR_INVALID_VALUE: invalid size, pointer, alignment or aliasing";
        case BTO_ERR_UNSUPPORTED: return "BTO_ERR_UNSUPPORTED: request not implemented by this library version";
        case BTO_ERR_WORKSPACE: return "BTO_ERR_WORKSPACE: workspace missing or too small";
        case BTO_ERR_CUDA: return "BTO_ERR_CUDA: a CUDA runtime call or kernel launch failed";
        case BTO_ERR_TIMEOUT: return "BTO_ERR_TIMEOUT: a bounded device-side wait expired";
        case BTO_ERR_BUDGET: return "BTO_ERR_BUDGET: request exceeds the configured memory budget";
        default: return "unknown bto status";
    }
}

extern "C" int bto_last_invalid_arg(void) { return last_invalid_arg(); }

extern "C" bto_status bto_device_status(const void* ws, bto_stream_t stream, int* status) {
    clear_invalid_arg();
    if (!ws) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (!status) { set_invalid_arg(3); return BTO_ERR_INVALID_VALUE; }
    int v = 0;
    if (cudaMemcpyAsync(&v, ws, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
        return BTO_ERR_CUDA;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return BTO_ERR_CUDA;
    *status = v;
    return BTO_OK;
}

extern "C" bto_status bto_workspace_bytes(int op, int form, int64_t m, int64_t n, int a_type,
                                          size_t* bytes) {
    clear_invalid_arg();
    if (op < BTO_OP_BICGK || op > BTO_OP_VADD) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (form < BTO_FORM_FUSED || form > BTO_FORM_DF_UNFUSED) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    if (m < 0) { set_invalid_arg(3); return BTO_ERR_INVALID_VALUE; }
    if (n < 0) { set_invalid_arg(4); return BTO_ERR_INVALID_VALUE; }
    if (a_type < BTO_F64 || a_type > BTO_BF16) { set_invalid_arg(5); return BTO_ERR_INVALID_VALUE; }
    if (!bytes) { set_invalid_arg(6); return BTO_ERR_INVALID_VALUE; }
    DeviceInfo d;
    if (!device_info(&d)) return BTO_ERR_CUDA;
    WsLayout L;
    bto_status st = ws_layout(op, form, m, n, a_type, d, &L);
    if (st != BTO_OK) return st;
    *bytes = L.total;
    return BTO_OK;
}
