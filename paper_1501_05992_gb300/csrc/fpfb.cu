// Fine polyphase filterbank: the second channeliser of the F stage (Section
// 3.2.1), a critically sampled n_taps-tap, 128-point filter-response-weighted
// DFT that splits each 1.28 MHz coarse channel into 128 fine channels of
// 10 kHz.  For coarse channel q, input i and frame m (one output sample per
// 128 input samples):
//
//     u_m[n] = sum_{p < n_taps} h[p * 128 + n] * x_qi[(m + p) * 128 + n]
//     Y_m[k] = sum_{n < 128} u_m[n] exp(-2 pi i k n / 128)
//
// and fine channel c = (k + 64) mod 128 (c = 0 the lowest frequency).  The
// window h is the caller's: the paper gives the structure, not the
// coefficients.  Output: the spectra as float pairs and/or their 4+4-bit codes
// clamp(rint(scale Y), -7, 7) (Appendix A: real part in the high nibble) in
// the X-engine's input layout [frame][q * 128 + c][input], so the F and X
// stages chain on the device.
//
// Work decomposition.  A CTA of 8 warps takes 8 consecutive inputs of one
// coarse channel over a run of frames; warp w owns input 8 blockIdx.x + w and
// lane l the points n = 4 l .. 4 l + 3 (one 8-byte load per lane covers a
// 128-sample block, coalesced).  Frames go in groups of G = 8: the G + n_taps - 1
// blocks that feed a group are loaded once each (from L1 for the n_taps - 1
// shared with the previous group), converted to float once, and each block is
// multiply-added into the accumulators of the frames it reaches (all register
// indices are compile-time, the block loop being unrolled).  The window sits
// in registers (4 n_taps per lane), the accumulators too (8 G per lane).
// The 128-point DFT of a frame is then done in the warp with n = 4 n1 + n2
// (n1 = lane, n2 = register j):
//
//     Y[k1 + 32 k2] = sum_{n2 < 4} W4^{n2 k2} W128^{n2 k1} sum_{n1 < 32} x[4 n1 + n2] W32^{n1 k1}
//
// i.e. four 32-point DIF transforms across lanes (shuffles; lane l ends with
// k1 = bitrev5(l)), a twiddle, and a 4-point DFT inside each lane.  The codes
// of a group go through shared memory so that each output row carries the 8
// inputs of the CTA together.
//
// The work is fp32 arithmetic (about 10.6 kflop per frame and input: 12 x 128
// complex-by-real multiply-adds and a 128-point FFT) against 256 bytes read and
// 128 bytes written, so the kernel is bound by the FP32 pipes, not by HBM.
#include "internal.cuh"

namespace corr {
namespace {

constexpr int kPfbPoints = 128;
constexpr int kPfbWarps = 8;                  // inputs per CTA
constexpr int kPfbThreads = kPfbWarps * 32;
constexpr int kPfbFramesPerCta = 120;         // frames per CTA (whole groups of 8)

struct PfbArgs {
    const int8_t *x;      // [Q][N][S][2]
    const float *h;       // [taps][128]
    uint8_t *volt;        // [M][Q * 128][N] or null
    float2 *spec;         // [M][Q * 128][N] or null
    long long S;          // samples per input
    int Q, N, M;          // coarse channels, inputs, frames
    float scale;
};

// signed bytes of w as floats: (s + 128) placed in the mantissa of 2^23, then
// 2^23 + 128 subtracted (exact for every byte)
__device__ __forceinline__ void bytes_to_float(uint32_t w, float &b0, float &b1, float &b2, float &b3)
{
    const uint32_t u = w ^ 0x80808080u;
    b0 = __int_as_float(int(__byte_perm(u, 0x4B000000u, 0x7440))) - 8388736.0f;
    b1 = __int_as_float(int(__byte_perm(u, 0x4B000000u, 0x7441))) - 8388736.0f;
    b2 = __int_as_float(int(__byte_perm(u, 0x4B000000u, 0x7442))) - 8388736.0f;
    b3 = __int_as_float(int(__byte_perm(u, 0x4B000000u, 0x7443))) - 8388736.0f;
}

__device__ __forceinline__ int quant4(float v)
{
    const int r = __float2int_rn(v);                  // round half to even
    return r > 7 ? 7 : (r < -7 ? -7 : r);
}

// exp(-2 pi i r / 128)
__device__ __forceinline__ float2 w128(int r)
{
    float s, c;
    sincospif(-float(r & 127) / 64.0f, &s, &c);
    return make_float2(c, s);
}

template <int TAPS, int G>
__global__ void __launch_bounds__(kPfbThreads, 1) fpfb_kernel(PfbArgs a)
{
    // G frames per group (kPfbFramesPerCta is a multiple of G); B blocks feed them
    static_assert(kPfbFramesPerCta % G == 0, "whole groups per CTA");
    constexpr int B = G + TAPS - 1;
    __shared__ __align__(16) uint8_t tile[G][kPfbPoints][kPfbWarps];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = blockIdx.z;
    const int i = blockIdx.x * kPfbWarps + warp;
    const bool active = i < a.N;
    const int m0 = blockIdx.y * kPfbFramesPerCta;
    const int m1 = min(a.M, m0 + kPfbFramesPerCta);
    const long long n_blocks = a.S / kPfbPoints;
    const size_t C = size_t(a.Q) * kPfbPoints;

    // the window at this lane's points, for every tap
    float hr[TAPS][4];
#pragma unroll
    for (int p = 0; p < TAPS; ++p) {
        const float4 v = *reinterpret_cast<const float4 *>(a.h + p * kPfbPoints + 4 * lane);
        hr[p][0] = v.x;
        hr[p][1] = v.y;
        hr[p][2] = v.z;
        hr[p][3] = v.w;
    }
    // twiddles: DIF stage with half span d uses W_{2d}^{l mod d} = W128^{(l mod d) 64 / d}
    // on the upper lane of each pair; after the transform lane l holds k1 = bitrev5(l)
    float2 tw[5];
    float sg[5];
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int d = 16 >> st;
        const bool upper = (lane & d) != 0;
        tw[st] = upper ? w128((lane & (d - 1)) * (64 / d)) : make_float2(1.0f, 0.0f);
        sg[st] = upper ? -1.0f : 1.0f;
    }
    const int k1 = __brev(unsigned(lane)) >> 27;
    const float2 t1 = w128(k1), t2 = w128(2 * k1), t3 = w128(3 * k1);

    const int8_t *xi = a.x + (size_t(q) * a.N + (active ? i : 0)) * size_t(a.S) * 2;

    for (int g0 = m0; g0 < m1; g0 += G) {
        float ar[G][4], am[G][4];
#pragma unroll
        for (int f = 0; f < G; ++f)
#pragma unroll
            for (int j = 0; j < 4; ++j) ar[f][j] = am[f][j] = 0.0f;
#pragma unroll
        for (int bb = 0; bb < B; ++bb) {
            const long long b = g0 + bb;
            uint2 w = make_uint2(0u, 0u);
            if (active && b < n_blocks)
                w = *reinterpret_cast<const uint2 *>(xi + (b * kPfbPoints + 4 * lane) * 2);
            float xr[4], xm[4];
            bytes_to_float(w.x, xr[0], xm[0], xr[1], xm[1]);
            bytes_to_float(w.y, xr[2], xm[2], xr[3], xm[3]);
#pragma unroll
            for (int p = 0; p < TAPS; ++p) {
                const int f = bb - p;                  // frame g0 + f takes this block as tap p
                if (f >= 0 && f < G) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        ar[f][j] = fmaf(hr[p][j], xr[j], ar[f][j]);
                        am[f][j] = fmaf(hr[p][j], xm[j], am[f][j]);
                    }
                }
            }
        }
#pragma unroll
        for (int f = 0; f < G; ++f) {
            const int m = g0 + f;
            if (m >= m1) break;                        // uniform across the CTA
            float zr[4], zm[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                zr[j] = ar[f][j];
                zm[j] = am[f][j];
            }
            // 32-point DIF across lanes, four transforms at once
#pragma unroll
            for (int st = 0; st < 5; ++st) {
                const int d = 16 >> st;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float vr = __shfl_xor_sync(0xffffffffu, zr[j], d);
                    const float vm = __shfl_xor_sync(0xffffffffu, zm[j], d);
                    // lower lane: own + partner; upper lane: (partner - own) * twiddle
                    const float sr = fmaf(sg[st], zr[j], vr), sm = fmaf(sg[st], zm[j], vm);
                    zr[j] = sr * tw[st].x - sm * tw[st].y;
                    zm[j] = sr * tw[st].y + sm * tw[st].x;
                }
            }
            // twiddle W128^{j k1}, then the 4-point DFT over j (W4 = -i)
            {
                float r, s;
                r = zr[1] * t1.x - zm[1] * t1.y; s = zr[1] * t1.y + zm[1] * t1.x; zr[1] = r; zm[1] = s;
                r = zr[2] * t2.x - zm[2] * t2.y; s = zr[2] * t2.y + zm[2] * t2.x; zr[2] = r; zm[2] = s;
                r = zr[3] * t3.x - zm[3] * t3.y; s = zr[3] * t3.y + zm[3] * t3.x; zr[3] = r; zm[3] = s;
            }
            const float e0r = zr[0] + zr[2], e0m = zm[0] + zm[2];
            const float e1r = zr[0] - zr[2], e1m = zm[0] - zm[2];
            const float o0r = zr[1] + zr[3], o0m = zm[1] + zm[3];
            const float o1r = zr[1] - zr[3], o1m = zm[1] - zm[3];
            float yr[4], ym[4];
            yr[0] = e0r + o0r; ym[0] = e0m + o0m;
            yr[2] = e0r - o0r; ym[2] = e0m - o0m;
            yr[1] = e1r + o1m; ym[1] = e1m - o1r;      // e1 - i o1
            yr[3] = e1r - o1m; ym[3] = e1m + o1r;      // e1 + i o1
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) {
                const int c = k1 + 32 * ((k2 + 2) & 3);   // (k1 + 32 k2 + 64) mod 128
                if (a.spec && active)
                    a.spec[(size_t(m) * C + size_t(q) * kPfbPoints + c) * a.N + i] = make_float2(yr[k2], ym[k2]);
                const int cr = quant4(yr[k2] * a.scale), cm = quant4(ym[k2] * a.scale);
                tile[f][c][warp] = uint8_t(((cr & 15) << 4) | (cm & 15));
            }
        }
        if (a.volt) {
            __syncthreads();
            const int nf = min(G, m1 - g0);
            const int i0 = blockIdx.x * kPfbWarps;
            const bool full = i0 + kPfbWarps <= a.N && (a.N & 7) == 0;
            for (int r = threadIdx.x; r < nf * kPfbPoints; r += kPfbThreads) {
                const int f = r / kPfbPoints, c = r % kPfbPoints;
                uint8_t *dst = a.volt + (size_t(g0 + f) * C + size_t(q) * kPfbPoints + c) * a.N + i0;
                if (full) {
                    *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<const uint2 *>(&tile[f][c][0]);
                } else {
                    for (int w = 0; w < kPfbWarps && i0 + w < a.N; ++w) dst[w] = tile[f][c][w];
                }
            }
            __syncthreads();
        }
    }
}

}  // namespace

cudaError_t launch_fine_pfb(const int8_t *x, int n_coarse, int n_inputs, long long n_samples, const float *window,
                            int n_taps, float scale, uint8_t *volt, float *spec, cudaStream_t s)
{
    PfbArgs a;
    a.x = x;
    a.h = window;
    a.volt = volt;
    a.spec = reinterpret_cast<float2 *>(spec);
    a.S = n_samples;
    a.Q = n_coarse;
    a.N = n_inputs;
    a.M = int(n_samples / kPfbPoints - n_taps + 1);
    a.scale = scale;
    const dim3 grid((n_inputs + kPfbWarps - 1) / kPfbWarps, (a.M + kPfbFramesPerCta - 1) / kPfbFramesPerCta, n_coarse);
    if (n_taps == 12)
        fpfb_kernel<12, 8><<<grid, kPfbThreads, 0, s>>>(a);
    else
        fpfb_kernel<1, 8><<<grid, kPfbThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace corr
