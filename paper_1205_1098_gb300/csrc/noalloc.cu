// bto_bicgk_noalloc: BICGK for callers that cannot allocate device memory.
//
// The split partial sums that bto_bicgk keeps in a caller-provided
// workspace live here in one file-scope device array of fixed size,
// reserved when the library's module is loaded on a device and held by that
// device until the process exits.  Host code must not use the array's name
// as a device address (on the host it names a host-side stand-in), so the
// real address is looked up once per device with cudaGetSymbolAddress and
// then passed to bto_bicgk as its workspace.  Nothing here allocates.
#include "check.cuh"
#include <mutex>
#include <vector>

namespace {

constexpr size_t kScratchBytes = (size_t)4 << 20;   // BTO_NOALLOC_SCRATCH_BYTES in bto.h

static __device__ __align__(256) unsigned char g_bicgk_scratch[kScratchBytes];

// Device address of g_bicgk_scratch on the current device, looked up on the
// first call made on that device.
bto_status scratch_address(void** out) {
    static std::mutex mu;
    static std::vector<void*> addr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BTO_ERR_CUDA;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)addr.size() <= dev) addr.resize(dev + 1, nullptr);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bicgk_scratch) != cudaSuccess || !p) return BTO_ERR_CUDA;
        addr[dev] = p;
    }
    *out = addr[dev];
    return BTO_OK;
}

}  // namespace

extern "C" bto_status bto_bicgk_noalloc(int64_t m, int64_t n, const double* A, int64_t lda,
                                        const double* p, const double* r, double* q, double* s,
                                        bto_stream_t stream) {
    bto::clear_invalid_arg();
    if (m < 0) { bto::set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (n < 0) { bto::set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    size_t need = 0;
    bto_status st = bto_workspace_bytes(BTO_OP_BICGK, BTO_FORM_FUSED, m, n, BTO_F64, &need);
    if (st != BTO_OK) return st;
    if (need > kScratchBytes) {
        // The problem's partial sums do not fit the fixed scratch array.
        bto::set_invalid_arg(m > n ? 1 : 2);
        return BTO_ERR_WORKSPACE;
    }
    void* ws = nullptr;
    if ((st = scratch_address(&ws)) != BTO_OK) return st;
    // Every scratch element the call reads is written earlier in the same
    // call, so the array needs no clearing between calls.
    return bto_bicgk(m, n, A, lda, p, r, q, s, ws, kScratchBytes, stream);
}
