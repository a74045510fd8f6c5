// Dump (K3): hand the integrated packed triangle to the caller.
//
// Section 3.4.3: products are accumulated on the device and then copied out;
// Appendix C ("GPU Output"): only the packed triangle with the autos leaves
// the GPU.  Every X-engine here already accumulates straight into the packed
// triangle layout int32 [f][i(i+1)/2 + j][2], so the dump is a streaming copy
// (or, for an integration with no samples, a zero fill).  Starting the next
// integration costs nothing: the context marks the accumulators "fresh" and
// the next X-engine launch stores instead of adding.
#include "internal.cuh"

namespace corr {
namespace {

__global__ void __launch_bounds__(256)
dump_copy_kernel(const int4 *__restrict__ src, int4 *__restrict__ dst, size_t n_vec)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n_vec;
         e += (size_t)gridDim.x * blockDim.x)
        dst[e] = __ldcs(src + e);
}

__global__ void __launch_bounds__(256)
dump_zero_kernel(int4 *__restrict__ dst, size_t n_vec)
{
    const int4 z = make_int4(0, 0, 0, 0);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n_vec;
         e += (size_t)gridDim.x * blockDim.x)
        dst[e] = z;
}

__global__ void dump_tail_kernel(const int32_t *src, int32_t *dst, size_t n, bool fresh)
{
    for (size_t e = threadIdx.x; e < n; e += blockDim.x) dst[e] = fresh ? 0 : src[e];
}

}  // namespace

cudaError_t launch_dump(const int32_t *acc, int32_t *vis, size_t n_words, bool fresh,
                        cudaStream_t s, int *launches)
{
    *launches = 0;
    if (n_words == 0) return cudaSuccess;
    const bool aligned = ((reinterpret_cast<uintptr_t>(acc) | reinterpret_cast<uintptr_t>(vis)) & 15) == 0;
    size_t n_vec = aligned ? n_words / 4 : 0;
    if (n_vec) {
        const int blocks = int(n_vec / 256 + 1 < 152 * 16 ? n_vec / 256 + 1 : 152 * 16);
        if (fresh)
            dump_zero_kernel<<<blocks, 256, 0, s>>>(reinterpret_cast<int4 *>(vis), n_vec);
        else
            dump_copy_kernel<<<blocks, 256, 0, s>>>(reinterpret_cast<const int4 *>(acc),
                                                    reinterpret_cast<int4 *>(vis), n_vec);
        ++*launches;
    }
    const size_t done = n_vec * 4;
    if (done < n_words) {
        dump_tail_kernel<<<1, 256, 0, s>>>(acc + done, vis + done, n_words - done, fresh);
        ++*launches;
    }
    return cudaGetLastError();
}

}  // namespace corr
