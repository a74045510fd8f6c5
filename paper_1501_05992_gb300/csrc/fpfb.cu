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
// 128-sample block, coalesced).  Frames go in groups of G = 4: the G + n_taps - 1
// blocks that feed a group are loaded once each (from L1 for the n_taps - 1
// shared with the previous group), converted to float once, and each block is
// multiply-added into the accumulators of the frames it reaches (all register
// indices are compile-time, the block loop being unrolled).  The window sits
// in registers (4 n_taps per lane), the accumulators too (8 G per lane), which
// keeps a thread at 128 registers: two CTAs (16 warps) per SM.  The lane's
// points are handled in pairs (j, j + 1) with the paired fp32 instructions of
// sm_100+ (fma/mul/add over a float2), which halves the instruction count of
// the windowing and of the butterflies.
// The 128-point DFT of a frame is then done in the warp with n = 4 n1 + n2
// (n1 = lane, n2 = register j):
//
//     Y[k1 + 32 k2] = sum_{n2 < 4} W4^{n2 k2} W128^{n2 k1} sum_{n1 < 32} x[4 n1 + n2] W32^{n1 k1}
//
// i.e. four 32-point DIF transforms across lanes (shuffles; lane l ends with
// k1 = bitrev5(l)), a twiddle, and a 4-point DFT inside each lane; two frames
// go through the transform together so that their shuffles and arithmetic
// interleave.  The codes of a group go through shared memory so that each
// output row carries the 8 inputs of the CTA together.
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
constexpr int kPfbFramesPerCta = 120;         // frames per CTA (whole groups of 4)

struct PfbArgs {
    const int8_t *x;      // [Q][N][S][2]
    const float *h;       // [taps][128]
    uint8_t *volt;        // [M][Q * 128][N] or null
    float2 *spec;         // [M][Q * 128][N] or null
    long long S;          // samples per input
    int Q, N, M;          // coarse channels, inputs, frames
    float scale;
};

// exp(-2 pi i r / 128)
__device__ __forceinline__ float2 w128(int r)
{
    float s, c;
    sincospif(-float(r & 127) / 64.0f, &s, &c);
    return make_float2(c, s);
}

// Paired fp32 arithmetic (sm_100+): one instruction does the two lanes of a float2.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

template <int TAPS, int G>
__global__ void __launch_bounds__(kPfbThreads, 2) fpfb_kernel(PfbArgs a)
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

    // Each lane's four points j = 0..3 are handled as two pairs (j, j + 1), so
    // that every multiply-add of the windowing and of the transforms is a
    // paired instruction over two points (or two transforms).
    // The window at this lane's points, for every tap: h2[p][0] = (h[4l], h[4l+1]), ...
    float2 h2[TAPS][2];
#pragma unroll
    for (int p = 0; p < TAPS; ++p) {
        const float4 v = *reinterpret_cast<const float4 *>(a.h + p * kPfbPoints + 4 * lane);
        h2[p][0] = make_float2(v.x, v.y);
        h2[p][1] = make_float2(v.z, v.w);
    }
    // twiddles: DIF stage with half span d uses W_{2d}^{l mod d} = W128^{(l mod d) 64 / d}
    // on the upper lane of each pair (1 on the lower); after the transform lane l
    // holds k1 = bitrev5(l).  Kept as duplicated pairs for the paired arithmetic.
    float2 sg2[5], wr2[5], wi2[5], nwi2[5];
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int d = 16 >> st;
        const bool upper = (lane & d) != 0;
        const float2 w = upper ? w128((lane & (d - 1)) * (64 / d)) : make_float2(1.0f, 0.0f);
        sg2[st] = dup2(upper ? -1.0f : 1.0f);
        wr2[st] = dup2(w.x);
        wi2[st] = dup2(w.y);
        nwi2[st] = dup2(-w.y);
    }
    const int k1 = __brev(unsigned(lane)) >> 27;
    // W128^{j k1} for j = 0..3, as pairs (j = 0, 1) and (j = 2, 3)
    const float2 t1 = w128(k1), t2 = w128(2 * k1), t3 = w128(3 * k1);
    const float2 tr01 = make_float2(1.0f, t1.x), ti01 = make_float2(0.0f, t1.y), nti01 = make_float2(0.0f, -t1.y);
    const float2 tr23 = make_float2(t2.x, t3.x), ti23 = make_float2(t2.y, t3.y), nti23 = make_float2(-t2.y, -t3.y);
    const float2 bias = dup2(-8388736.0f), minus1 = dup2(-1.0f), scale2 = dup2(a.scale), magic2 = dup2(12582912.0f);

    const int8_t *xi = a.x + (size_t(q) * a.N + (active ? i : 0)) * size_t(a.S) * 2;

    for (int g0 = m0; g0 < m1; g0 += G) {
        // ar[f][h] = real parts of frame g0 + f at points (2h, 2h + 1) of this lane; am imaginary
        float2 ar[G][2], am[G][2];
#pragma unroll
        for (int f = 0; f < G; ++f)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) ar[f][hh] = am[f][hh] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int bb = 0; bb < B; ++bb) {
            const long long b = g0 + bb;
            uint2 w = make_uint2(0u, 0u);
            if (active && b < n_blocks)
                w = *reinterpret_cast<const uint2 *>(xi + (b * kPfbPoints + 4 * lane) * 2);
            // bytes (re0, im0, re1, im1 | re2, im2, re3, im3) -> floats; the signed
            // byte s becomes 2^23 + s + 128 in the float's mantissa, then the bias goes
            const uint32_t u0 = w.x ^ 0x80808080u, u1 = w.y ^ 0x80808080u;
            float2 xr[2], xm[2];
            xr[0] = add2(make_float2(__int_as_float(int(__byte_perm(u0, 0x4B000000u, 0x7440))),
                                     __int_as_float(int(__byte_perm(u0, 0x4B000000u, 0x7442)))), bias);
            xm[0] = add2(make_float2(__int_as_float(int(__byte_perm(u0, 0x4B000000u, 0x7441))),
                                     __int_as_float(int(__byte_perm(u0, 0x4B000000u, 0x7443)))), bias);
            xr[1] = add2(make_float2(__int_as_float(int(__byte_perm(u1, 0x4B000000u, 0x7440))),
                                     __int_as_float(int(__byte_perm(u1, 0x4B000000u, 0x7442)))), bias);
            xm[1] = add2(make_float2(__int_as_float(int(__byte_perm(u1, 0x4B000000u, 0x7441))),
                                     __int_as_float(int(__byte_perm(u1, 0x4B000000u, 0x7443)))), bias);
#pragma unroll
            for (int p = 0; p < TAPS; ++p) {
                const int f = bb - p;                  // frame g0 + f takes this block as tap p
                if (f >= 0 && f < G) {
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        ar[f][hh] = fma2(h2[p][hh], xr[hh], ar[f][hh]);
                        am[f][hh] = fma2(h2[p][hh], xm[hh], am[f][hh]);
                    }
                }
            }
        }
#pragma unroll
        for (int f0 = 0; f0 < G; f0 += 2) {
            if (g0 + f0 >= m1) break;                  // uniform across the CTA
            float2 zr[2][2], zm[2][2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                zr[u][0] = ar[f0 + u][0]; zr[u][1] = ar[f0 + u][1];
                zm[u][0] = am[f0 + u][0]; zm[u][1] = am[f0 + u][1];
            }
#pragma unroll
            for (int st = 0; st < 5; ++st) {
                const int d = 16 >> st;
                float2 vr[2][2], vm[2][2];
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        vr[u][hh] = make_float2(__shfl_xor_sync(0xffffffffu, zr[u][hh].x, d),
                                                __shfl_xor_sync(0xffffffffu, zr[u][hh].y, d));
                        vm[u][hh] = make_float2(__shfl_xor_sync(0xffffffffu, zm[u][hh].x, d),
                                                __shfl_xor_sync(0xffffffffu, zm[u][hh].y, d));
                    }
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const float2 sr = fma2(sg2[st], zr[u][hh], vr[u][hh]), sm = fma2(sg2[st], zm[u][hh], vm[u][hh]);
                        zr[u][hh] = fma2(sm, nwi2[st], mul2(sr, wr2[st]));
                        zm[u][hh] = fma2(sm, wr2[st], mul2(sr, wi2[st]));
                    }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int f = f0 + u, m = g0 + f;
                {
                    const float2 r0 = fma2(zm[u][0], nti01, mul2(zr[u][0], tr01)), s0 = fma2(zm[u][0], tr01, mul2(zr[u][0], ti01));
                    const float2 r1 = fma2(zm[u][1], nti23, mul2(zr[u][1], tr23)), s1 = fma2(zm[u][1], tr23, mul2(zr[u][1], ti23));
                    zr[u][0] = r0; zm[u][0] = s0; zr[u][1] = r1; zm[u][1] = s1;
                }
                const float2 eor = add2(zr[u][0], zr[u][1]), eom = add2(zm[u][0], zm[u][1]);
                const float2 e1r_o1r = fma2(zr[u][1], minus1, zr[u][0]), e1m_o1m = fma2(zm[u][1], minus1, zm[u][0]);
                float2 y[4];
                y[0] = make_float2(eor.x + eor.y, eom.x + eom.y);
                y[2] = make_float2(eor.x - eor.y, eom.x - eom.y);
                y[1] = make_float2(e1r_o1r.x + e1m_o1m.y, e1m_o1m.x - e1r_o1r.y);
                y[3] = make_float2(e1r_o1r.x - e1m_o1m.y, e1m_o1m.x + e1r_o1r.y);
#pragma unroll
                for (int k2 = 0; k2 < 4; ++k2) {
                    const int c = k1 + 32 * ((k2 + 2) & 3);
                    if (a.spec && active && m < m1)
                        a.spec[(size_t(m) * C + size_t(q) * kPfbPoints + c) * a.N + i] = y[k2];
                    // clamp to [-7, 7], then adding 1.5 * 2^23 rounds to the nearest
                    // integer, ties to even, and leaves it (two's complement) in the
                    // low mantissa bits
                    const float2 v = mul2(y[k2], scale2);
                    const float2 w = add2(make_float2(fminf(fmaxf(v.x, -7.0f), 7.0f), fminf(fmaxf(v.y, -7.0f), 7.0f)),
                                          magic2);
                    tile[f][c][warp] = uint8_t(((__float_as_uint(w.x) & 15u) << 4) | (__float_as_uint(w.y) & 15u));
                }
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
        fpfb_kernel<12, 4><<<grid, kPfbThreads, 0, s>>>(a);
    else
        fpfb_kernel<1, 4><<<grid, kPfbThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace corr
