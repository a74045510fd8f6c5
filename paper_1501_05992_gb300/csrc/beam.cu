// Incoherent beam: total power of all inputs per channel and sample.
//
// Section 3.4 lists incoherent beam forming among the XMAC's modes beside the
// correlation: the power sum over every input of a channel, at the voltage
// time resolution (or integrated over n_avg samples):
//
//     beam[k][f] = sum over the n_avg samples t of block k, over inputs n, of |x_n(t,f)|^2
//
// One thread owns one channel of one output sample and walks the N input
// bytes of each of its n_avg rows in 16-byte chunks.  Per 32-bit word (four
// inputs) the real and imaginary nibbles are sign-extended into signed bytes
// and one dp4a of each with itself adds four squares.  The kernel is bound by
// HBM reads (N bytes per sample and channel); rows of neighbouring channels
// are adjacent, so a warp's loads cover whole cache lines over its chunks.
#include "internal.cuh"

namespace corr {
namespace {

constexpr int kBeamThreads = 128;

// |x|^2 of the four samples in w, summed (4-bit two's complement nibbles, real
// in the high nibble).  With zero_invalid a sample with either nibble 8
// contributes nothing.
template <bool kZeroInvalid>
__device__ __forceinline__ int power4(uint32_t w, int acc)
{
    const uint32_t uh = ((w >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;   // code + 8, 0..15
    const uint32_t ul = (w & 0x0F0F0F0Fu) ^ 0x08080808u;
    uint32_t vh = __vsub4(uh, 0x08080808u);                       // signed bytes -8..7
    uint32_t vl = __vsub4(ul, 0x08080808u);
    if (kZeroInvalid) {
        // a nibble code 8 has u == 0; zero both parts of such samples
        const uint32_t bad = __vcmpeq4(uh, 0u) | __vcmpeq4(ul, 0u);
        vh &= ~bad;
        vl &= ~bad;
    }
    acc = __dp4a(int(vh), int(vh), acc);
    return __dp4a(int(vl), int(vl), acc);
}

template <bool kZeroInvalid, bool kVec>
__global__ void __launch_bounds__(kBeamThreads)
beam_kernel(const uint8_t *__restrict__ volt, int n, int n_chan, int n_avg, int n_out, int32_t *__restrict__ out)
{
    const int f = blockIdx.x * kBeamThreads + threadIdx.x;
    if (f >= n_chan) return;
    for (int k = blockIdx.y; k < n_out; k += gridDim.y) {
    int acc = 0;
    for (int t = k * n_avg; t < (k + 1) * n_avg; ++t) {
        const uint8_t *row = volt + ((size_t)t * n_chan + f) * n;
        if (kVec) {
            for (int c = 0; c < n; c += 16) {
                const uint4 w = *reinterpret_cast<const uint4 *>(row + c);
                acc = power4<kZeroInvalid>(w.x, acc);
                acc = power4<kZeroInvalid>(w.y, acc);
                acc = power4<kZeroInvalid>(w.z, acc);
                acc = power4<kZeroInvalid>(w.w, acc);
            }
        } else {
            // one sample per word; the three zero bytes are valid samples of value 0
            for (int c = 0; c < n; ++c) acc = power4<kZeroInvalid>(uint32_t(row[c]), acc);
        }
    }
    out[(size_t)k * n_chan + f] = acc;
    }
}

}  // namespace

cudaError_t launch_beam(const uint8_t *volt, int n_time, int n_chan, int n, int n_avg, bool zero_invalid,
                        int32_t *out, cudaStream_t s)
{
    const int n_out = n_time / n_avg;
    if (n_out == 0) return cudaSuccess;
    const bool vec = n % 16 == 0 && (reinterpret_cast<uintptr_t>(volt) & 15) == 0;
    const dim3 grid(unsigned(div_up(n_chan, kBeamThreads)), unsigned(n_out < 65535 ? n_out : 65535));
    if (zero_invalid) {
        if (vec) beam_kernel<true, true><<<grid, kBeamThreads, 0, s>>>(volt, n, n_chan, n_avg, n_out, out);
        else beam_kernel<true, false><<<grid, kBeamThreads, 0, s>>>(volt, n, n_chan, n_avg, n_out, out);
    } else {
        if (vec) beam_kernel<false, true><<<grid, kBeamThreads, 0, s>>>(volt, n, n_chan, n_avg, n_out, out);
        else beam_kernel<false, false><<<grid, kBeamThreads, 0, s>>>(volt, n, n_chan, n_avg, n_out, out);
    }
    return cudaGetLastError();
}

}  // namespace corr
