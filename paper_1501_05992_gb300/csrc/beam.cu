// Incoherent beam: total power of all inputs per channel and sample.
//
// Section 3.4 lists incoherent beam forming among the XMAC's modes beside the
// correlation: the power sum over every input of a channel, at the voltage
// time resolution (or integrated over n_avg samples):
//
//     beam[k][f] = sum over the n_avg samples t of block k, over inputs n, of |x_n(t,f)|^2
//
// The kernel is bound by HBM reads (N bytes per sample and channel, 4 bytes
// written per output).  Where N is a multiple of 16 a group of L lanes (L the
// largest power of two up to 32 dividing N / 16) reads one channel's row of a
// sample, each lane 16-byte chunks L chunks apart, so a warp's load covers
// 32 / L neighbouring rows, i.e. 512 contiguous bytes; the group adds its
// lanes' sums with shuffles once per output.  A block takes 128 neighbouring
// channels (32 KB per sample at N = 256).  Per 32-bit word (four samples) the
// high nibbles with the low ones cleared are the signed bytes 16 r, the low
// nibbles moved up 16 m, and two dp4a add 256 (r^2 + m^2); each row's sum is
// divided by 256 before it is added, which keeps every partial sum within
// int32 wherever the result is.  Other input counts take one thread per
// channel and output, walking the row byte by byte.
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

// One thread per channel and output; one sample per word (the three zero bytes
// are valid samples of value 0).
template <bool kZeroInvalid>
__global__ void __launch_bounds__(kBeamThreads)
beam_bytes_kernel(const uint8_t *__restrict__ volt, int n, int n_chan, int n_avg, int n_out,
                  int32_t *__restrict__ out)
{
    const int f = blockIdx.x * kBeamThreads + threadIdx.x;
    if (f >= n_chan) return;
    for (int k = blockIdx.y; k < n_out; k += gridDim.y) {
        int acc = 0;
        for (int t = k * n_avg; t < (k + 1) * n_avg; ++t) {
            const uint8_t *row = volt + ((size_t)t * n_chan + f) * n;
            for (int c = 0; c < n; ++c) acc = power4<kZeroInvalid>(uint32_t(row[c]), acc);
        }
        out[(size_t)k * n_chan + f] = acc;
    }
}

// 256 (r^2 + m^2) summed over the four samples of w, plus acc (the high nibble
// with the low one cleared is the signed byte 16 r; the low nibble moved up,
// 16 m).  With zero_invalid a sample with either nibble 8 contributes nothing.
template <bool kZeroInvalid>
__device__ __forceinline__ int power4x256(uint32_t w, int acc)
{
    uint32_t hr = w & 0xF0F0F0F0u, hm = (w << 4) & 0xF0F0F0F0u;
    if (kZeroInvalid) {
        const uint32_t bad = __vcmpeq4(hr, 0x80808080u) | __vcmpeq4(hm, 0x80808080u);
        hr &= ~bad;
        hm &= ~bad;
    }
    return __dp4a(int(hm), int(hm), __dp4a(int(hr), int(hr), acc));
}

constexpr int kBeamRowThreads = 256;
constexpr int kBeamBlockChans = 128;

// kL lanes per channel row (N a multiple of 16 kL; 16-byte aligned rows).  A
// thread takes kU of its group's channels at a time, so that kU loads (per
// chunk) are in flight before the first is used.
template <bool kZeroInvalid, int kL>
__global__ void __launch_bounds__(kBeamRowThreads)
beam_rows_kernel(const uint8_t *__restrict__ volt, int n, int n_chan, int n_avg, int n_out,
                 int32_t *__restrict__ out)
{
    constexpr int kGroups = kBeamRowThreads / kL;
    constexpr int kChans = kGroups > kBeamBlockChans ? kGroups : kBeamBlockChans;
    constexpr int kIter = kChans / kGroups;
    constexpr int kU = kIter < 4 ? kIter : 4;
    const int sub = threadIdx.x % kL, group = threadIdx.x / kL;
    const int per_lane = n / (16 * kL);
    const int f0 = blockIdx.x * kChans;
    for (int k = blockIdx.y; k < n_out; k += gridDim.y) {
        // the trip counts are the same for every group, so whole warps shuffle
        for (int fb = group; fb < kChans; fb += kU * kGroups) {
            int acc[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) acc[u] = 0;
            for (int t = k * n_avg; t < (k + 1) * n_avg; ++t) {
                const uint4 *row[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    // a channel past the end reads channel 0's row and is not stored
                    const int f = f0 + fb + u * kGroups;
                    row[u] = reinterpret_cast<const uint4 *>(volt + ((size_t)t * n_chan + (f < n_chan ? f : 0)) * n) +
                             sub;
                }
                int p[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) p[u] = 0;
                for (int j = 0; j < per_lane; ++j) {
                    uint4 w[kU];
#pragma unroll
                    for (int u = 0; u < kU; ++u) w[u] = row[u][j * kL];
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        p[u] = power4x256<kZeroInvalid>(w[u].x, p[u]);
                        p[u] = power4x256<kZeroInvalid>(w[u].y, p[u]);
                        p[u] = power4x256<kZeroInvalid>(w[u].z, p[u]);
                        p[u] = power4x256<kZeroInvalid>(w[u].w, p[u]);
                    }
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) acc[u] += p[u] >> 8;
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
#pragma unroll
                for (int o = kL / 2; o >= 1; o /= 2) acc[u] += __shfl_xor_sync(0xFFFFFFFFu, acc[u], o);
                const int f = f0 + fb + u * kGroups;
                if (sub == 0 && f < n_chan) out[(size_t)k * n_chan + f] = acc[u];
            }
        }
    }
}

template <bool kZeroInvalid>
cudaError_t launch_rows(int lanes, const uint8_t *volt, int n, int n_chan, int n_avg, int n_out, int32_t *out,
                        cudaStream_t s)
{
    const int groups = kBeamRowThreads / lanes;
    const int chans = groups > kBeamBlockChans ? groups : kBeamBlockChans;
    // a few outputs per block: 1024 rows of blocks at most
    const dim3 grid(unsigned(div_up(n_chan, chans)), unsigned(n_out < 1024 ? n_out : 1024));
    switch (lanes) {
    case 1: beam_rows_kernel<kZeroInvalid, 1><<<grid, kBeamRowThreads, 0, s>>>(volt, n, n_chan, n_avg, n_out, out); break;
    case 2: beam_rows_kernel<kZeroInvalid, 2><<<grid, kBeamRowThreads, 0, s>>>(volt, n, n_chan, n_avg, n_out, out); break;
    case 4: beam_rows_kernel<kZeroInvalid, 4><<<grid, kBeamRowThreads, 0, s>>>(volt, n, n_chan, n_avg, n_out, out); break;
    case 8: beam_rows_kernel<kZeroInvalid, 8><<<grid, kBeamRowThreads, 0, s>>>(volt, n, n_chan, n_avg, n_out, out); break;
    case 16: beam_rows_kernel<kZeroInvalid, 16><<<grid, kBeamRowThreads, 0, s>>>(volt, n, n_chan, n_avg, n_out, out); break;
    default: beam_rows_kernel<kZeroInvalid, 32><<<grid, kBeamRowThreads, 0, s>>>(volt, n, n_chan, n_avg, n_out, out); break;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_beam(const uint8_t *volt, int n_time, int n_chan, int n, int n_avg, bool zero_invalid,
                        int32_t *out, cudaStream_t s)
{
    const int n_out = n_time / n_avg;
    if (n_out == 0) return cudaSuccess;
    if (n % 16 == 0 && (reinterpret_cast<uintptr_t>(volt) & 15) == 0) {
        // lanes per row: the largest power of two up to 32 dividing the row's chunks
        const int chunks = n / 16;
        int lanes = 1;
        while (lanes < 32 && chunks % (2 * lanes) == 0) lanes *= 2;
        return zero_invalid ? launch_rows<true>(lanes, volt, n, n_chan, n_avg, n_out, out, s)
                            : launch_rows<false>(lanes, volt, n, n_chan, n_avg, n_out, out, s);
    }
    const dim3 grid(unsigned(div_up(n_chan, kBeamThreads)), unsigned(n_out < 65535 ? n_out : 65535));
    if (zero_invalid) beam_bytes_kernel<true><<<grid, kBeamThreads, 0, s>>>(volt, n, n_chan, n_avg, n_out, out);
    else beam_bytes_kernel<false><<<grid, kBeamThreads, 0, s>>>(volt, n, n_chan, n_avg, n_out, out);
    return cudaGetLastError();
}

}  // namespace corr
