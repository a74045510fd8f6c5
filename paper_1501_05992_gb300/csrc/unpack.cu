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

// r, m and -m of the four packed samples of w, as four signed bytes each.  With
// u = nibble ^ 8 = value + 8 (0..15) in every byte, (u + 0x78) ^ 0x80 is the
// signed byte u - 8 and (0x88 - u) ^ 0x80 the signed byte 8 - u, and neither sum
// carries out of its byte.  A zero byte gives 0 + 0i.
__device__ __forceinline__ void decode4(uint32_t w, bool zero_invalid, uint32_t &R, uint32_t &M, uint32_t &N)
{
    const uint32_t ur = ((w >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
    const uint32_t um = (w & 0x0F0F0F0Fu) ^ 0x08080808u;
    R = (ur + 0x78787878u) ^ 0x80808080u;
    M = (um + 0x78787878u) ^ 0x80808080u;
    N = (0x88888888u - um) ^ 0x80808080u;
    if (zero_invalid) {
        // a nibble code of 8 (u == 0) in either part makes the sample 0 + 0i
        const uint32_t bad = __vcmpeq4(ur, 0u) | __vcmpeq4(um, 0u);
        R &= ~bad;
        M &= ~bad;
        N &= ~bad;
    }
}

// Byte k of X and byte k of Y for k = 0..3, interleaved as two words:
// lo = (X0, Y0, X1, Y1), hi = (X2, Y2, X3, Y3).
__device__ __forceinline__ void zip4(uint32_t X, uint32_t Y, uint32_t &lo, uint32_t &hi)
{
    lo = __byte_perm(X, Y, 0x5140);
    hi = __byte_perm(X, Y, 0x7362);
}

// From A = (a0, b0, a1, b1) and B = (c0, d0, c1, d1): (a0, b0, c0, d0) and (a1, b1, c1, d1).
__device__ __forceinline__ void pairs2(uint32_t A, uint32_t B, uint32_t &first, uint32_t &second)
{
    first = __byte_perm(A, B, 0x5410);
    second = __byte_perm(A, B, 0x7632);
}

// Four inputs' words (r(t), m(t), r(t+1), m(t+1)) and their twisted copies
// (-m(t), r(t), -m(t+1), r(t+1)) from the packed samples of the four inputs at
// t (w0) and t + 1 (w1).
__device__ __forceinline__ void words4(uint32_t w0, uint32_t w1, bool zero_invalid, uint32_t wa[4], uint32_t ww[4])
{
    uint32_t R0, M0, N0, R1, M1, N1;
    decode4(w0, zero_invalid, R0, M0, N0);
    decode4(w1, zero_invalid, R1, M1, N1);
    uint32_t a0, a1, b0, b1;
    zip4(R0, M0, a0, a1);
    zip4(R1, M1, b0, b1);
    pairs2(a0, b0, wa[0], wa[1]);
    pairs2(a1, b1, wa[2], wa[3]);
    zip4(N0, R0, a0, a1);
    zip4(N1, R1, b0, b1);
    pairs2(a0, b0, ww[0], ww[1]);
    pairs2(a1, b1, ww[2], ww[3]);
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
        const uint8_t *base = volt + (long long)(f0 + fl) * n + n0;
        uint32_t wa[G], ww[G];
        if (G == 4) {
            // n % 4 == 0: four inputs of a group are all real or all padding;
            // padding and samples past nt are zero bytes, i.e. 0 + 0i
            uint32_t w0 = 0, w1 = 0;
            if (n0 < n && t0 < nt) w0 = __ldg(reinterpret_cast<const uint32_t *>(base + t0 * row_stride));
            if (n0 < n && t0 + 1 < nt) w1 = __ldg(reinterpret_cast<const uint32_t *>(base + (t0 + 1) * row_stride));
            words4(w0, w1, zero_invalid, wa, ww);
        } else {
#pragma unroll
            for (int k = 0; k < G; ++k) {
                const bool v0 = (n0 + k < n) && (t0 < nt), v1 = (n0 + k < n) && (t0 + 1 < nt);
                int r0, m0, r1, m1;
                decode_byte(v0 ? base[t0 * row_stride + k] : 0u, zero_invalid, r0, m0);
                decode_byte(v1 ? base[(t0 + 1) * row_stride + k] : 0u, zero_invalid, r1, m1);
                wa[k] = pack4(r0, m0, r1, m1);
                ww[k] = pack4(-m0, r0, -m1, r1);
            }
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

// K-major: a 64-sample x 64-input tile per block, staged in shared memory with
// loads coalesced along inputs (16 bytes a thread where rows allow).  A thread
// then takes 4 inputs x 4 samples: four 32-bit reads of the tile (one per
// sample, four inputs each), the SIMD decode, and byte permutes that turn them
// into each input's 8 bytes (r, m) x 4 samples and its twisted 8 bytes; the
// 16 threads of an input group write 128 contiguous bytes per input.
constexpr int kKT = 64, kKN = 64, kKPitchW = 17;   // tile row: 64 bytes + one pad word

__global__ void __launch_bounds__(256)
unpack_kmajor_kernel(const uint8_t *__restrict__ volt, int n_chan, int n, int f0,
                     int nt, int n_pad, int t_pad, bool zero_invalid, bool vec16,
                     int8_t *__restrict__ out, int8_t *__restrict__ out_tw)
{
    __shared__ uint32_t tile[kKT * kKPitchW];
    const int fl = blockIdx.z;
    const int nb = blockIdx.y * kKN;
    const int tb = blockIdx.x * kKT;
    const long long row_stride = (long long)n_chan * n;
    const uint8_t *base = volt + (long long)(f0 + fl) * n;
    if (vec16) {
        // n % 16 == 0 and 16-byte aligned rows: a 16-byte piece is all inputs or all padding
        const int tt = threadIdx.x >> 2, q = threadIdx.x & 3;
        const int t = tb + tt, ni = nb + 16 * q;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (t < nt && ni < n) v = __ldg(reinterpret_cast<const uint4 *>(base + t * row_stride + ni));
        uint32_t *row = tile + tt * kKPitchW + 4 * q;
        row[0] = v.x;
        row[1] = v.y;
        row[2] = v.z;
        row[3] = v.w;
    } else {
        uint8_t *t8 = reinterpret_cast<uint8_t *>(tile);
        for (int e = threadIdx.x; e < kKT * kKN; e += blockDim.x) {
            const int tt = e / kKN, nn = e % kKN;
            const int t = tb + tt, ni = nb + nn;
            t8[tt * (4 * kKPitchW) + nn] = (t < nt && ni < n) ? base[t * row_stride + ni] : 0;
        }
    }
    __syncthreads();
    const int tg = threadIdx.x & 15, ig = threadIdx.x >> 4;
    uint32_t R[4], M[4], N[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) decode4(tile[(4 * tg + s) * kKPitchW + ig], zero_invalid, R[s], M[s], N[s]);
    // lo[k] = (r, m) of samples 0, 1 of input k, hi[k] of samples 2, 3; tl, th twisted
    uint32_t lo[4], hi[4], tl[4], th[4], a0, a1, b0, b1;
    zip4(R[0], M[0], a0, a1);
    zip4(R[1], M[1], b0, b1);
    pairs2(a0, b0, lo[0], lo[1]);
    pairs2(a1, b1, lo[2], lo[3]);
    zip4(R[2], M[2], a0, a1);
    zip4(R[3], M[3], b0, b1);
    pairs2(a0, b0, hi[0], hi[1]);
    pairs2(a1, b1, hi[2], hi[3]);
    zip4(N[0], R[0], a0, a1);
    zip4(N[1], R[1], b0, b1);
    pairs2(a0, b0, tl[0], tl[1]);
    pairs2(a1, b1, tl[2], tl[3]);
    zip4(N[2], R[2], a0, a1);
    zip4(N[3], R[3], b0, b1);
    pairs2(a0, b0, th[0], th[1]);
    pairs2(a1, b1, th[2], th[3]);
    const int t = tb + 4 * tg;
    if (t >= t_pad) return;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int ni = nb + 4 * ig + k;
        if (ni >= n_pad) break;
        const long long o = (((long long)fl * n_pad + ni) * t_pad + t) * 2;
        int8_t *dst = out + o;
        if (t + 4 <= t_pad && (reinterpret_cast<uintptr_t>(dst) & 7) == 0) {
            *reinterpret_cast<uint2 *>(dst) = make_uint2(lo[k], hi[k]);
        } else {
            const uint32_t v[2] = {lo[k], hi[k]};
            for (int j = 0; j < 8 && t + j / 2 < t_pad; ++j) dst[j] = int8_t(v[j / 4] >> (8 * (j % 4)));
        }
        if (out_tw) {
            int8_t *dtw = out_tw + o;
            if (t + 4 <= t_pad && (reinterpret_cast<uintptr_t>(dtw) & 7) == 0) {
                *reinterpret_cast<uint2 *>(dtw) = make_uint2(tl[k], th[k]);
            } else {
                const uint32_t v[2] = {tl[k], th[k]};
                for (int j = 0; j < 8 && t + j / 2 < t_pad; ++j) dtw[j] = int8_t(v[j / 4] >> (8 * (j % 4)));
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

// dst[row * ld + x] = src[row * n + x] for x < n (and 0 for n <= x < ld): one
// thread per 16-byte piece of a destination row, written with one store; the
// source is read four bytes at a time where n % 4 == 0 (rows then start on
// 4-byte boundaries), else byte by byte.
template <bool kWords, typename Index>
__global__ void __launch_bounds__(256)
pad_rows_kernel(const uint8_t *__restrict__ src, Index rows, int n, int ld, uint8_t *__restrict__ dst)
{
    const Index pieces = Index(ld / 16);
    const Index total = rows * pieces;
    for (Index e = Index(blockIdx.x) * 256 + threadIdx.x; e < total; e += Index(gridDim.x) * 256) {
        const Index row = e / pieces;
        const int b0 = 16 * int(e - row * pieces);
        const uint8_t *s = src + (long long)row * n + b0;
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int x = b0 + 4 * k;
            if (kWords) {
                w[k] = x < n ? __ldg(reinterpret_cast<const uint32_t *>(s + 4 * k)) : 0u;
            } else {
                w[k] = 0u;
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (x + b < n) w[k] |= uint32_t(__ldg(s + 4 * k + b)) << (8 * b);
            }
        }
        *reinterpret_cast<uint4 *>(dst + (long long)row * ld + b0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

}  // namespace

cudaError_t launch_pad_rows(const uint8_t *src, long long rows, int n, int ld, uint8_t *dst, cudaStream_t s)
{
    if (rows <= 0 || n <= 0) return cudaSuccess;
    if (ld % 16 != 0 || (reinterpret_cast<uintptr_t>(dst) & 15) != 0) return cudaErrorInvalidValue;
    const long long total = rows * (ld / 16);
    const long long want = (total + 255) / 256;
    const int blocks = int(want < 152 * 16 ? want : 152 * 16);
    const bool words = n % 4 == 0 && (reinterpret_cast<uintptr_t>(src) & 3) == 0;
    if (total < (1LL << 31) - (1LL << 21)) {   // an int index and its grid stride cannot overflow
        if (words) pad_rows_kernel<true, int><<<blocks, 256, 0, s>>>(src, int(rows), n, ld, dst);
        else pad_rows_kernel<false, int><<<blocks, 256, 0, s>>>(src, int(rows), n, ld, dst);
    } else {
        if (words) pad_rows_kernel<true, long long><<<blocks, 256, 0, s>>>(src, rows, n, ld, dst);
        else pad_rows_kernel<false, long long><<<blocks, 256, 0, s>>>(src, rows, n, ld, dst);
    }
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
    const bool vec16 = n % 16 == 0 && (reinterpret_cast<uintptr_t>(volt) & 15) == 0;
    unpack_kmajor_kernel<<<grid, 256, 0, s>>>(volt, n_chan, n, f0, nt, n_pad, t_pad,
                                              zero_invalid, vec16, out, out_tw);
    return cudaGetLastError();
}

}  // namespace corr
