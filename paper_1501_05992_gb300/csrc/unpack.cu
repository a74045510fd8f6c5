// Unpack + corner turn (K1).
//
// The paper does this on the XMAC host: the receiver threads transpose the
// PFB's mixed time/frequency order into time, channel, station, polarisation,
// complex order and promote each 4-bit component to 8 bits through a lookup
// table so that the GPU can widen 8 -> 32 bits cheaply (Section 3.4.1;
// Appendix C, "GPU Input").  Here the GPU does it, straight from the packed
// 4+4-bit bytes (Appendix A "Data Format": real = high nibble, imaginary = low
// nibble, two's complement), writing the operand layout each X-engine wants:
//
//   words  : A[f][tw][n] = (r(2tw), m(2tw), r(2tw+1), m(2tw+1)) int8x4 and the
//            "twisted" plane W[f][tw][n] = (-m, r, -m, r) for the dp4a kernel,
//            inputs contiguous so that one 16-byte load feeds four inputs;
//   K-major: X[f][n][t][2] int8 (time contiguous per input) for mma.sync,
//            optionally with its twisted plane Xt[f][n][t][2] = (-m, r).
//
// Both are HBM-bound: one byte read and 4 (words: 2 planes x 2 bytes) or 2
// (K-major) bytes written per complex sample.
//
// The tensor-core path reads the packed bytes themselves, through TMA, which
// needs rows (the n inputs of one channel and sample) that start on 16-byte
// boundaries.  For other input counts the rows are first copied to a stride
// of round_up(n, 16) bytes (the bytes between rows are never read: the
// tensor map's extent is n and TMA fills columns past it with zeros).
#include "internal.cuh"

namespace corr {
namespace {

__device__ __forceinline__ void decode_byte(uint32_t b, bool zero_invalid, int &r, int &m)
{
    r = ((int)(int8_t)(uint8_t)b) >> 4;             // high nibble, sign-extended
    m = ((int)(int8_t)(uint8_t)(b << 4)) >> 4;      // low nibble, sign-extended
    if (zero_invalid && (((b & 0xF0u) == 0x80u) || ((b & 0x0Fu) == 0x08u))) {
        r = 0;
        m = 0;
    }
}

__device__ __forceinline__ uint32_t pack4(int a, int b, int c, int d)
{
    return (uint32_t(a) & 0xFFu) | ((uint32_t(b) & 0xFFu) << 8) |
           ((uint32_t(c) & 0xFFu) << 16) | ((uint32_t(d) & 0xFFu) << 24);
}

// One thread per (channel, word, group of G inputs).  G = 4 uses one 32-bit
// load per sample row (needs n % 4 == 0 and a 4-byte aligned base).
template <int G>
__global__ void __launch_bounds__(256)
unpack_words_kernel(const uint8_t *__restrict__ volt, int n_chan, int n, int f0, int fc,
                    int nt, int n_pad, int tw_pad, bool zero_invalid,
                    int32_t *__restrict__ A, int32_t *__restrict__ W)
{
    const int groups = n_pad / G;
    const long long total = (long long)fc * tw_pad * groups;
    const long long row_stride = (long long)n_chan * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int g = int(e % groups);
        const long long rest = e / groups;
        const int tw = int(rest % tw_pad);
        const int fl = int(rest / tw_pad);
        const int n0 = g * G;
        const int t0 = 2 * tw;
        uint32_t b0[G], b1[G];
        bool v0[G], v1[G];
        const uint8_t *base = volt + (long long)(f0 + fl) * n + n0;
        if (G == 4 && n0 + 3 < n) {
            uint32_t w0 = 0, w1 = 0;
            if (t0 < nt) w0 = __ldg(reinterpret_cast<const uint32_t *>(base + t0 * row_stride));
            if (t0 + 1 < nt) w1 = __ldg(reinterpret_cast<const uint32_t *>(base + (t0 + 1) * row_stride));
#pragma unroll
            for (int k = 0; k < G; ++k) {
                b0[k] = (w0 >> (8 * k)) & 0xFFu;
                b1[k] = (w1 >> (8 * k)) & 0xFFu;
                v0[k] = t0 < nt;
                v1[k] = t0 + 1 < nt;
            }
        } else {
#pragma unroll
            for (int k = 0; k < G; ++k) {
                v0[k] = (n0 + k < n) && (t0 < nt);
                v1[k] = (n0 + k < n) && (t0 + 1 < nt);
                b0[k] = v0[k] ? base[t0 * row_stride + k] : 0u;
                b1[k] = v1[k] ? base[(t0 + 1) * row_stride + k] : 0u;
            }
        }
        uint32_t wa[G], ww[G];
#pragma unroll
        for (int k = 0; k < G; ++k) {
            int r0, m0, r1, m1;
            decode_byte(b0[k], zero_invalid, r0, m0);
            decode_byte(b1[k], zero_invalid, r1, m1);
            if (!v0[k]) { r0 = 0; m0 = 0; }
            if (!v1[k]) { r1 = 0; m1 = 0; }
            wa[k] = pack4(r0, m0, r1, m1);
            ww[k] = pack4(-m0, r0, -m1, r1);
        }
        const long long o = ((long long)fl * tw_pad + tw) * n_pad + n0;
        if (G == 4) {
            *reinterpret_cast<uint4 *>(A + o) = make_uint4(wa[0], wa[1], wa[2], wa[3]);
            *reinterpret_cast<uint4 *>(W + o) = make_uint4(ww[0], ww[1], ww[2], ww[3]);
        } else {
#pragma unroll
            for (int k = 0; k < G; ++k) {
                A[o + k] = int32_t(wa[k]);
                W[o + k] = int32_t(ww[k]);
            }
        }
    }
}

// K-major: a 64-sample x 64-input tile per block, transposed through shared
// memory.  Reads are coalesced along inputs, writes along time.
constexpr int kKT = 64, kKN = 64, kKPad = 65;

__global__ void __launch_bounds__(256)
unpack_kmajor_kernel(const uint8_t *__restrict__ volt, int n_chan, int n, int f0,
                     int nt, int n_pad, int t_pad, bool zero_invalid,
                     int8_t *__restrict__ out, int8_t *__restrict__ out_tw)
{
    __shared__ uint8_t tile[kKT][kKPad];
    __shared__ uint8_t valid[kKT][kKPad];
    const int fl = blockIdx.z;
    const int nb = blockIdx.y * kKN;
    const int tb = blockIdx.x * kKT;
    const long long row_stride = (long long)n_chan * n;
    const uint8_t *base = volt + (long long)(f0 + fl) * n;
    for (int e = threadIdx.x; e < kKT * kKN; e += blockDim.x) {
        const int tt = e / kKN, nn = e % kKN;
        const int t = tb + tt, ni = nb + nn;
        const bool ok = t < nt && ni < n;
        tile[tt][nn] = ok ? base[t * row_stride + ni] : 0;
        valid[tt][nn] = ok;
    }
    __syncthreads();
    // each thread writes 4 consecutive samples (8 bytes) of one input
    for (int e = threadIdx.x; e < kKN * (kKT / 4); e += blockDim.x) {
        const int nn = e / (kKT / 4), tg = e % (kKT / 4);
        const int ni = nb + nn;
        if (ni >= n_pad) continue;
        int v[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int r, m;
            decode_byte(tile[tg * 4 + k][nn], zero_invalid, r, m);
            if (!valid[tg * 4 + k][nn]) { r = 0; m = 0; }
            v[2 * k] = r;
            v[2 * k + 1] = m;
        }
        const int t = tb + tg * 4;
        if (t >= t_pad) continue;
        int8_t *dst = out + (((long long)fl * n_pad + ni) * t_pad + t) * 2;
        const uint32_t lo = pack4(v[0], v[1], v[2], v[3]);
        const uint32_t hi = pack4(v[4], v[5], v[6], v[7]);
        if (t + 4 <= t_pad && ((reinterpret_cast<uintptr_t>(dst) & 7) == 0)) {
            *reinterpret_cast<uint2 *>(dst) = make_uint2(lo, hi);
        } else {
            for (int k = 0; k < 8 && t + k / 2 < t_pad; ++k)
                dst[k] = int8_t(v[k]);
        }
        if (out_tw) {
            // twisted plane (-m, r): dot((r_i, m_i), (-m_j, r_j)) = m_i r_j - r_i m_j
            int8_t *dtw = out_tw + (((long long)fl * n_pad + ni) * t_pad + t) * 2;
            const uint32_t tlo = pack4(-v[1], v[0], -v[3], v[2]);
            const uint32_t thi = pack4(-v[5], v[4], -v[7], v[6]);
            if (t + 4 <= t_pad && ((reinterpret_cast<uintptr_t>(dtw) & 7) == 0)) {
                *reinterpret_cast<uint2 *>(dtw) = make_uint2(tlo, thi);
            } else {
                const int tv[8] = {-v[1], v[0], -v[3], v[2], -v[5], v[4], -v[7], v[6]};
                for (int k = 0; k < 8 && t + k / 2 < t_pad; ++k)
                    dtw[k] = int8_t(tv[k]);
            }
        }
    }
}

int grid_for(long long total, int threads)
{
    long long b = (total + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152LL * 64) b = 152LL * 64;
    return int(b);
}

// dst[row * ld + x] = src[row * n + x] for x < n: one thread per source byte,
// reads and writes both coalesced along the row.
__global__ void __launch_bounds__(256)
pad_rows_kernel(const uint8_t *__restrict__ src, long long n_bytes, int n, int ld, uint8_t *__restrict__ dst)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n_bytes;
         e += (long long)gridDim.x * blockDim.x) {
        const long long row = e / n;
        dst[row * ld + (e - row * n)] = __ldg(src + e);
    }
}

}  // namespace

cudaError_t launch_pad_rows(const uint8_t *src, long long rows, int n, int ld, uint8_t *dst, cudaStream_t s)
{
    const long long n_bytes = rows * n;
    if (n_bytes <= 0) return cudaSuccess;
    const long long want = (n_bytes + 255) / 256;
    const int blocks = int(want < 152 * 32 ? want : 152 * 32);
    pad_rows_kernel<<<blocks, 256, 0, s>>>(src, n_bytes, n, ld, dst);
    return cudaGetLastError();
}

cudaError_t launch_unpack_words(const uint8_t *volt, int n_chan, int n, int f0, int fc,
                                int nt, int n_pad, int tw_pad, bool zero_invalid,
                                int32_t *A, int32_t *W, cudaStream_t s)
{
    const bool vec = (n % 4 == 0) && (n_pad % 4 == 0) &&
                     ((reinterpret_cast<uintptr_t>(volt) & 3) == 0);
    if (vec) {
        const long long total = (long long)fc * tw_pad * (n_pad / 4);
        unpack_words_kernel<4><<<grid_for(total, 256), 256, 0, s>>>(
            volt, n_chan, n, f0, fc, nt, n_pad, tw_pad, zero_invalid, A, W);
    } else {
        const long long total = (long long)fc * tw_pad * n_pad;
        unpack_words_kernel<1><<<grid_for(total, 256), 256, 0, s>>>(
            volt, n_chan, n, f0, fc, nt, n_pad, tw_pad, zero_invalid, A, W);
    }
    return cudaGetLastError();
}

cudaError_t launch_unpack_kmajor(const uint8_t *volt, int n_chan, int n, int f0, int fc,
                                 int nt, int n_pad, int t_pad, bool zero_invalid,
                                 int8_t *out, int8_t *out_tw, cudaStream_t s)
{
    if (fc <= 0 || t_pad <= 0 || n_pad <= 0) return cudaSuccess;
    dim3 grid(div_up(t_pad, kKT), div_up(n_pad, kKN), fc);
    unpack_kmajor_kernel<<<grid, 256, 0, s>>>(volt, n_chan, n, f0, nt, n_pad, t_pad,
                                              zero_invalid, out, out_tw);
    return cudaGetLastError();
}

}  // namespace corr
