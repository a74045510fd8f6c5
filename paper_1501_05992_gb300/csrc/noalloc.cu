// corr_xmac_noalloc: the CUDA-core X-engine for callers that cannot allocate
// device memory.
//
// Some callers are not allowed to call cudaMalloc at all once they are
// running: hosts that hand out every byte of device memory from their own
// pool and forbid allocations behind their back, and real-time acquisition
// loops in which an allocation (which may synchronise the device) would stall
// the data stream.  corr_create/corr_bind_workspace need a caller-allocated
// workspace; this entry point needs none.  Its scratch (the unpacked operand
// planes) lives in one statically sized __device__ array.  The CUDA runtime
// reserves it on a GPU when it loads the library's device code there: with
// lazy module loading (the default) that happens inside the first call on
// that device, whose symbol lookup below loads the module, so the first call
// can take device memory and synchronise.  Callers that must never do that
// once data flows make one warm-up call first (n_time == 0 is enough).  The
// array then stays reserved until the process exits.
//
// The caller still provides the voltages and the visibility buffer.  One call
// correlates one block as a whole integration and overwrites d_vis.
#include <mutex>

#include "internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(CORR_NOALLOC_SCRATCH_BYTES);
constexpr int kMaxDevices = 64;

// Shared by every call on a device; the unpack kernel rewrites every byte a
// call reads (padding included) before the X-engine reads it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on `dev` (which must be current).  The
// array's name in host code is only a stand-in for the symbol, so the real
// address is looked up once per device and cached.
int scratch_for(int dev, void **out)
{
    if (dev < 0 || dev >= kMaxDevices) return CORR_E_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return CORR_E_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return CORR_OK;
}

}  // namespace

extern "C" int corr_xmac_noalloc(const uint8_t *d_volt, int n_time, int n_chan, int n_inputs,
                                 int32_t *d_vis, unsigned flags, void *stream)
{
    using namespace corr;
    if (n_time < 0 || n_chan < 1 || n_chan > 65535 || n_inputs < 1 || n_inputs > 8192 ||
        (long long)n_time * 128LL >= (1LL << 31) || (flags & ~CORR_ZERO_INVALID) || !d_vis ||
        (n_time > 0 && !d_volt))
        return set_last_error(CORR_E_ARG);
    const int n_pad = int(round_up(size_t(n_inputs), kDp4aTile));
    const int tw_pad = int(round_up(size_t(n_time), 2 * kDp4aKW) / 2);
    const size_t plane = size_t(n_chan) * size_t(tw_pad) * size_t(n_pad);  // int32 words
    if (2 * plane * sizeof(int32_t) > kScratchBytes) return set_last_error(CORR_E_BUDGET);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return set_last_error(CORR_E_CUDA);
    }
    void *scratch = nullptr;
    const int rc = scratch_for(dev, &scratch);
    if (rc != CORR_OK) return set_last_error(rc);

    int32_t *A = static_cast<int32_t *>(scratch);
    int32_t *W = A + plane;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool zi = (flags & CORR_ZERO_INVALID) != 0;
    if (launch_unpack_words(d_volt, n_chan, n_inputs, 0, n_chan, n_time, n_pad, tw_pad, zi, A, W,
                            s) != cudaSuccess ||
        launch_xeng_dp4a(A, W, n_inputs, n_pad, n_chan, tw_pad, d_vis, 0, /*fresh=*/true, kDp4aTile, s) !=
            cudaSuccess)
        return set_last_error(CORR_E_CUDA);
    return set_last_error(CORR_OK);
}
