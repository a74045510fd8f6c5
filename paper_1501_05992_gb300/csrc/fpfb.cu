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
// Work decomposition.  A CTA of 4 warps takes 16 consecutive inputs of one
// coarse channel over a run of frames: frames in groups of G = 8, inputs in
// sub-batches of 2, so that one unit (group, sub-batch) is 16 (frame, input)
// transforms, taken in three phases separated by CTA barriers.
//
//  1. Windowing.  Warp w takes input w / 2 of the sub-batch and the points
//     64 (w mod 2) .. + 63, lane l the pair of points (2 l, 2 l + 1) of that
//     half (one 4-byte load per lane and block, 128 bytes per warp).  The
//     G + n_taps - 1 blocks that feed a unit are each loaded once, converted to
//     float once and multiply-added into the accumulators of the frames they
//     reach; the window sits in registers (one float pair per tap), and every
//     multiply-add is a paired fp32 instruction (sm_100+) over the lane's two
//     points.  The blocks of the next unit are loaded into registers before
//     this unit's transforms, so that the loads complete behind them.  The
//     windowed frames go to shared memory, real and imaginary planes apart.
//  2. 8-point DFTs.  With n = n1 + 16 n2 and k = k2 + 8 k1,
//
//       Y[k2 + 8 k1] = sum_{n1 < 16} W16^{n1 k1} W128^{n1 k2} sum_{n2 < 8} u[n1 + 16 n2] W8^{n2 k2},
//
//     a thread takes one transform and the two columns n1 = 2 r, 2 r + 1 as
//     the two halves of its float pairs (adjacent points: one 8-byte load per
//     pair), does the 8-point DFT over n2 in registers and applies
//     W128^{n1 k2} (a shared-memory table).
//  3. 16-point DFTs.  A thread takes one transform and one k2: its 16 values
//     over n1 arrive as 8 float pairs (even n1, odd n1), so the two 8-point
//     DFTs of the even and odd halves are paired instructions and the last
//     radix-2 step (W16^{k1}) is scalar.  The 16 outputs are clamped, rounded
//     and packed into codes in a shared-memory tile of the CTA's 16 inputs.
//  4. After the last sub-batch of a group, each output row piece (one frame,
//     one fine channel, the CTA's 16 inputs: 16 bytes) is written with one
//     16-byte store.  Scattered stores of a few bytes per row cost the store
//     path one transaction each, which is why a CTA gathers 16 inputs.
//
// No lane exchanges data with another through shuffles: the two transposes
// go through shared memory, laid out so that every access takes the minimum
// number of wavefronts for its width.  When only codes are written, the code
// scale rides on the W128 twiddles.
//
// The work is fp32 arithmetic (about 10.6 kflop per frame and input: 12 x 128
// complex-by-real multiply-adds and a 128-point FFT) against 256 bytes read and
// 128 bytes written, so the kernel is bound by the FP32 pipes, not by HBM.
#include <algorithm>

#include "internal.cuh"

namespace corr {
namespace {

constexpr int kPfbPoints = 128;
constexpr int kPfbThreads = 128;              // 4 warps
constexpr int kPfbSub = 2;                    // inputs per sub-batch, two windowing warps each
constexpr int kPfbInputs = 16;                // inputs per CTA: 8 sub-batches
constexpr int kPfbGroup = 8;                  // frames per group
constexpr int kPfbXf = kPfbSub * kPfbGroup;   // transforms per unit
constexpr int kPfbMaxFramesPerCta = 120;      // frames per CTA (whole groups), at most
constexpr int kPfbCtasPerSm = 4;
// shared memory: windowed frames [16][Re 128 | Im 128 | pad 16] floats (the
// pad spreads the transforms over the banks), 8-point results [16 transforms]
// [8 k2 rows of 8 float4 | pad 16 bytes], the W128 twiddles [8 k2][8 r]
// float4, and the codes [G frames][128 channels][16 inputs] bytes with the
// frame stride padded by 16 bytes
constexpr int kUStride = 2 * kPfbPoints + 16;             // floats
constexpr int kZStride = 8 * 8 * 4 + 4;                   // floats
constexpr int kTileFrame = kPfbPoints * kPfbInputs + 16;  // bytes
constexpr size_t kPfbSmem = sizeof(float) * (kPfbXf * kUStride + kPfbXf * kZStride + 8 * 8 * 4) +
                            size_t(kPfbGroup) * kTileFrame;

struct PfbArgs {
    const int8_t *x;      // [Q][N][S][2]
    const float *h;       // [taps][128]
    uint8_t *volt;        // [M][Q * 128][N] or null
    float2 *spec;         // [M][Q * 128][N] or null
    long long S;          // samples per input
    int Q, N, M;          // coarse channels, inputs, frames
    int fpc;              // frames per CTA (a multiple of the group)
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
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, dup2(-1.0f), a); }

// A complex value in each half of a float pair: two independent transforms.
struct C2 {
    float2 r, i;
};

// In-place 4-point DFT (W4 = -i) of x0..x3 on both halves.
__device__ __forceinline__ void dft4(C2 &x0, C2 &x1, C2 &x2, C2 &x3)
{
    const float2 s02r = add2(x0.r, x2.r), s02i = add2(x0.i, x2.i);
    const float2 d02r = sub2(x0.r, x2.r), d02i = sub2(x0.i, x2.i);
    const float2 s13r = add2(x1.r, x3.r), s13i = add2(x1.i, x3.i);
    const float2 d13r = sub2(x1.r, x3.r), d13i = sub2(x1.i, x3.i);
    x0.r = add2(s02r, s13r);
    x0.i = add2(s02i, s13i);
    x2.r = sub2(s02r, s13r);
    x2.i = sub2(s02i, s13i);
    x1.r = add2(d02r, d13i);            // d02 - i d13
    x1.i = sub2(d02i, d13r);
    x3.r = sub2(d02r, d13i);            // d02 + i d13
    x3.i = add2(d02i, d13r);
}

// In-place 8-point DFT (W8 = exp(-2 pi i / 8)) on both halves, radix-2 by
// frequency: t0[n] = x[n] + x[n + 4], t1[n] = (x[n] - x[n + 4]) W8^n, then
// X[2 k] = DFT4(t0)[k] lands in x[k] and X[2 k + 1] = DFT4(t1)[k] in x[k + 4].
__device__ __forceinline__ void dft8(C2 (&x)[8])
{
    const float2 H = dup2(0.70710678118654752f);
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        const C2 a = x[n], b = x[n + 4];
        x[n].r = add2(a.r, b.r);
        x[n].i = add2(a.i, b.i);
        x[n + 4].r = sub2(a.r, b.r);
        x[n + 4].i = sub2(a.i, b.i);
    }
    {   // W8 = (1 - i) / sqrt 2
        const float2 a = x[5].r, b = x[5].i;
        x[5].r = mul2(add2(a, b), H);
        x[5].i = mul2(sub2(b, a), H);
    }
    {   // W8^2 = -i
        const float2 a = x[6].r;
        x[6].r = x[6].i;
        x[6].i = mul2(a, dup2(-1.0f));
    }
    {   // W8^3 = -(1 + i) / sqrt 2
        const float2 a = x[7].r, b = x[7].i;
        x[7].r = mul2(sub2(b, a), H);
        x[7].i = mul2(add2(a, b), dup2(-0.70710678118654752f));
    }
    dft4(x[0], x[1], x[2], x[3]);
    dft4(x[4], x[5], x[6], x[7]);
}

template <int NB>
__device__ __forceinline__ void load_blocks(uint32_t (&w)[NB], const int8_t *x, long long b0, long long n_blocks,
                                            bool active)
{
#pragma unroll
    for (int bb = 0; bb < NB; ++bb) {
        const long long b = b0 + bb;
        w[bb] = active && b < n_blocks ? *reinterpret_cast<const uint32_t *>(x + b * (2 * kPfbPoints)) : 0u;
    }
}

template <int TAPS, bool kSpec, bool kVolt>
__global__ void __launch_bounds__(kPfbThreads, kPfbCtasPerSm) fpfb_kernel(PfbArgs a)
{
    constexpr int G = kPfbGroup;
    constexpr int B = G + TAPS - 1;             // blocks that feed a group
    static_assert(kPfbMaxFramesPerCta % G == 0, "whole groups per CTA");
    extern __shared__ __align__(16) float smem[];
    float *const U = smem;                                    // [32][kUStride]
    float *const Z = U + kPfbXf * kUStride;                   // [32][kZStride]
    float4 *const TW = reinterpret_cast<float4 *>(Z + kPfbXf * kZStride);   // [8][8]
    uint8_t *const tile = reinterpret_cast<uint8_t *>(TW + 8 * 8);          // [G][kTileFrame]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = blockIdx.z;
    const int i0 = blockIdx.x * kPfbInputs;
    const int n_sub = min(kPfbInputs, a.N - i0 + kPfbSub - 1) / kPfbSub;   // sub-batches with an input
    const int iw = warp >> 1;                   // windowing: this warp's input of a sub-batch, and half
    const int p0 = 64 * (warp & 1) + 2 * lane;
    const int m0 = blockIdx.y * a.fpc;
    const int m1 = min(a.M, m0 + a.fpc);
    const long long n_blocks = a.S / kPfbPoints;
    const size_t C = size_t(a.Q) * kPfbPoints;

    // W128^{n1 k2} for the two columns n1 = 2 r, 2 r + 1 of an 8-point thread,
    // (Re pair, Im pair) per (k2, r); times the code scale when only codes are
    // written, the scale then riding on the twiddles
    constexpr bool kFold = kVolt && !kSpec;
    const float tws = kFold ? a.scale : 1.0f;
    if (threadIdx.x < 64) {
        const int k2 = threadIdx.x >> 3, r = threadIdx.x & 7;
        const float2 w0 = w128(2 * r * k2), w1 = w128((2 * r + 1) * k2);
        TW[threadIdx.x] = make_float4(w0.x * tws, w1.x * tws, w0.y * tws, w1.y * tws);
    }
    // the window at this lane's two points, for every tap
    float2 h2[TAPS];
#pragma unroll
    for (int p = 0; p < TAPS; ++p) h2[p] = *reinterpret_cast<const float2 *>(a.h + p * kPfbPoints + p0);
    const float2 bias = dup2(-8388736.0f);
    auto stream = [&](int sb) {                 // this warp's input stream in sub-batch sb
        const int i = i0 + sb * kPfbSub + iw;
        return a.x + (size_t(q) * a.N + (i < a.N ? i : 0)) * size_t(a.S) * 2 + 2 * p0;
    };
    // the blocks of the first unit (group, sub-batch); every unit loads those
    // of the next one before its transforms, so that the loads complete behind them
    uint32_t wblk[B];
    load_blocks(wblk, stream(0), m0, n_blocks, i0 + iw < a.N);
    __syncthreads();

    for (int g0 = m0; g0 < m1; g0 += G) {
#pragma unroll 1
        for (int sb = 0; sb < n_sub; ++sb) {
            // ---- 1. windowing: ar[f] / am[f] = Re / Im of frame g0 + f at points (p0, p0 + 1)
            {
                float2 ar[G], am[G];
#pragma unroll
                for (int f = 0; f < G; ++f) ar[f] = am[f] = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int bb = 0; bb < B; ++bb) {
                    // bytes (re0, im0, re1, im1) -> floats: the signed byte s becomes
                    // 2^23 + s + 128 in the float's mantissa, then the bias goes
                    const uint32_t u = wblk[bb] ^ 0x80808080u;
                    const float2 xr = add2(make_float2(__int_as_float(int(__byte_perm(u, 0x4B000000u, 0x7440))),
                                                       __int_as_float(int(__byte_perm(u, 0x4B000000u, 0x7442)))),
                                           bias);
                    const float2 xm = add2(make_float2(__int_as_float(int(__byte_perm(u, 0x4B000000u, 0x7441))),
                                                       __int_as_float(int(__byte_perm(u, 0x4B000000u, 0x7443)))),
                                           bias);
#pragma unroll
                    for (int p = 0; p < TAPS; ++p) {
                        const int f = bb - p;           // frame g0 + f takes this block as tap p
                        if (f >= 0 && f < G) {
                            ar[f] = fma2(h2[p], xr, ar[f]);
                            am[f] = fma2(h2[p], xm, am[f]);
                        }
                    }
                }
#pragma unroll
                for (int f = 0; f < G; ++f) {
                    float *u = U + (iw * G + f) * kUStride + p0;
                    *reinterpret_cast<float2 *>(u) = ar[f];
                    *reinterpret_cast<float2 *>(u + kPfbPoints) = am[f];
                }
                // the next unit: the next sub-batch of this group, else the first of the next group
                const bool more = sb + 1 < n_sub;
                if (more || g0 + G < m1) {
                    const int nsb = more ? sb + 1 : 0;
                    load_blocks(wblk, stream(nsb), more ? g0 : g0 + G, n_blocks, i0 + nsb * kPfbSub + iw < a.N);
                }
            }
            __syncthreads();
            // ---- 2. 8-point DFTs over n2 (transform t / 8, columns n1 = 2 r, 2 r + 1)
            {
                const int xf = threadIdx.x >> 3, r = threadIdx.x & 7;
                const float *u = U + xf * kUStride + 2 * r;
                C2 x[8];
#pragma unroll
                for (int n2 = 0; n2 < 8; ++n2) {
                    x[n2].r = *reinterpret_cast<const float2 *>(u + 16 * n2);
                    x[n2].i = *reinterpret_cast<const float2 *>(u + kPfbPoints + 16 * n2);
                }
                dft8(x);                        // X[2 k] in x[k], X[2 k + 1] in x[k + 4]
                float4 *z = reinterpret_cast<float4 *>(Z + xf * kZStride);
#pragma unroll
                for (int k2 = 0; k2 < 8; ++k2) {
                    C2 v = x[(k2 >> 1) + 4 * (k2 & 1)];
                    if (k2 > 0) {
                        const float4 w = TW[k2 * 8 + r];
                        const float2 wr = make_float2(w.x, w.y), wi = make_float2(w.z, w.w);
                        const float2 vr = sub2(mul2(v.r, wr), mul2(v.i, wi));
                        v.i = fma2(v.r, wi, mul2(v.i, wr));
                        v.r = vr;
                    } else if (kFold) {
                        v.r = mul2(v.r, dup2(tws));
                        v.i = mul2(v.i, dup2(tws));
                    }
                    // row k2 (128 bytes), slot r ^ k2: 8 consecutive k2 of one slot cover all banks
                    z[k2 * 8 + (r ^ k2)] = make_float4(v.r.x, v.r.y, v.i.x, v.i.y);
                }
            }
            __syncthreads();
            // ---- 3. 16-point DFTs over n1 (warp k2, lane = transform)
            {
                const int xf = lane & 15, k2 = 2 * warp + (lane >> 4);
                const float4 *z = reinterpret_cast<const float4 *>(Z + xf * kZStride) + k2 * 8;
                C2 e[8];                        // .x: n1 = 2 r (even), .y: n1 = 2 r + 1 (odd)
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const float4 v = z[r ^ k2];
                    e[r].r = make_float2(v.x, v.y);
                    e[r].i = make_float2(v.z, v.w);
                }
                dft8(e);                        // E[k] (.x) and O[k] (.y): k even in e[k / 2], odd in e[4 + k / 2]
                const int iw3 = xf / G, f = xf % G, m = g0 + f, i = i0 + sb * kPfbSub + iw3;
                // Y[k2 + 8 k1] = E[k1] + W16^{k1} O[k1], Y[k2 + 8 (k1 + 8)] = E[k1] - W16^{k1} O[k1]
                const float c16 = 0.92387953251128674f, s16 = 0.38268343236508977f, h = 0.70710678118654752f;
                const float wre[8] = {1.0f, c16, h, s16, 0.0f, -s16, -h, -c16};
                const float wim[8] = {0.0f, -s16, -h, -c16, -1.0f, -c16, -h, -s16};
#pragma unroll
                for (int k1 = 0; k1 < 8; ++k1) {
                    const C2 &v = e[(k1 >> 1) + 4 * (k1 & 1)];
                    const float Er = v.r.x, Ei = v.i.x, Or = v.r.y, Oi = v.i.y;
                    float orr, oi;
                    if (k1 == 0) {
                        orr = Or;
                        oi = Oi;
                    } else if (k1 == 4) {
                        orr = Oi;
                        oi = -Or;
                    } else if (k1 == 2 || k1 == 6) {
                        orr = (k1 == 2 ? Or + Oi : Oi - Or) * h;
                        oi = (k1 == 2 ? Oi - Or : -(Or + Oi)) * h;
                    } else {
                        orr = fmaf(Or, wre[k1], -Oi * wim[k1]);
                        oi = fmaf(Or, wim[k1], Oi * wre[k1]);
                    }
#pragma unroll
                    for (int hi = 0; hi < 2; ++hi) {
                        const float yr = hi ? Er - orr : Er + orr, yi = hi ? Ei - oi : Ei + oi;
                        const int c = (k2 + 8 * (k1 + 8 * hi) + 64) & 127;
                        if (kSpec && i < a.N && m < m1)
                            a.spec[(size_t(m) * C + size_t(q) * kPfbPoints + c) * a.N + i] = make_float2(yr, yi);
                        if (kVolt) {
                            // clamp to [-7, 7], then adding 1.5 * 2^23 rounds to the nearest
                            // integer, ties to even, and leaves it (two's complement) in the
                            // low mantissa bits
                            const float2 s = kFold ? make_float2(yr, yi) : mul2(make_float2(yr, yi), dup2(a.scale));
                            const float2 w = add2(make_float2(fminf(fmaxf(s.x, -7.0f), 7.0f),
                                                              fminf(fmaxf(s.y, -7.0f), 7.0f)), dup2(12582912.0f));
                            tile[f * kTileFrame + c * kPfbInputs + sb * kPfbSub + iw3] =
                                uint8_t((__float_as_uint(w.x) << 4) | (__float_as_uint(w.y) & 15u));
                        }
                    }
                }
            }
            // the next unit writes U after its windowing (every 8-point load of
            // this unit came before the second barrier above) and Z after its
            // first barrier (every 16-point load of this unit comes before it)
        }
        if (kVolt) {
            // ---- 4. the group's codes, one 32-byte row piece (32 inputs) per output row
            __syncthreads();
            const int nf = min(G, m1 - g0);
            const bool full = i0 + kPfbInputs <= a.N && (a.N & 15) == 0 &&
                              (reinterpret_cast<uintptr_t>(a.volt) & 15) == 0;
            constexpr int kChunks = kPfbInputs / 16;
            for (int t = threadIdx.x; t < nf * kPfbPoints * kChunks; t += kPfbThreads) {
                const int row = t / kChunks, hh = t % kChunks, f = row / kPfbPoints, c = row % kPfbPoints;
                uint8_t *dst = a.volt + (size_t(g0 + f) * C + size_t(q) * kPfbPoints + c) * a.N + i0 + 16 * hh;
                const uint8_t *src = tile + f * kTileFrame + c * kPfbInputs + 16 * hh;
                if (full) {
                    *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(src);
                } else {
                    for (int w = 0; w < 16 && i0 + 16 * hh + w < a.N; ++w) dst[w] = src[w];
                }
            }
            // the next group writes the codes only after two more barriers,
            // which every thread reaches after its copy-out
        }
    }
}

constexpr int kPfbMaxDevices = 64;

template <int TAPS, bool kSpec, bool kVolt>
cudaError_t launch_pfb(const PfbArgs &a, dim3 grid, int dev, cudaStream_t s)
{
    // the attributes belong to each device's copy of the kernel: set once per
    // device (setting them twice is harmless); all of the shared memory the SM
    // has, since the blocks each unit re-reads come from L2 and registers
    static bool configured[kPfbMaxDevices] = {};
    if (dev >= kPfbMaxDevices || !configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(fpfb_kernel<TAPS, kSpec, kVolt>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(kPfbSmem));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fpfb_kernel<TAPS, kSpec, kVolt>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        if (dev < kPfbMaxDevices) configured[dev] = true;
    }
    fpfb_kernel<TAPS, kSpec, kVolt><<<grid, kPfbThreads, kPfbSmem, s>>>(a);
    return cudaGetLastError();
}

template <int TAPS>
cudaError_t launch_taps(const PfbArgs &a, dim3 grid, int dev, cudaStream_t s)
{
    if (a.spec && a.volt) return launch_pfb<TAPS, true, true>(a, grid, dev, s);
    if (a.spec) return launch_pfb<TAPS, true, false>(a, grid, dev, s);
    return launch_pfb<TAPS, false, true>(a, grid, dev, s);
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
    // frames per CTA: the longest run (fewest CTA prologues) that still gives
    // two waves of CTAs over the SMs
    static int sm_count[kPfbMaxDevices] = {};
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < kPfbMaxDevices && sm_count[dev] > 0) {
        sms = sm_count[dev];
    } else {
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        if (dev < kPfbMaxDevices) sm_count[dev] = sms;
    }
    const long long gx = (n_inputs + kPfbInputs - 1) / kPfbInputs;
    const long long want = 2LL * sms * kPfbCtasPerSm;
    const long long per_cta = (a.M * gx * n_coarse + want - 1) / want;
    a.fpc = int(std::min<long long>(kPfbMaxFramesPerCta,
                                    std::max<long long>(kPfbGroup, (per_cta + kPfbGroup - 1) / kPfbGroup * kPfbGroup)));
    const dim3 grid(unsigned(gx), unsigned((a.M + a.fpc - 1) / a.fpc), unsigned(n_coarse));
    return n_taps == 12 ? launch_taps<12>(a, grid, dev, s) : launch_taps<1>(a, grid, dev, s);
}

}  // namespace corr
