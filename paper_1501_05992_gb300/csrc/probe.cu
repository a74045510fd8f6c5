// Throughput probes: the peak rates the X-engine kernels are measured
// against, taken on the device in the same run instead of assumed.
//
//   tcgen05 FP8   tcgen05.mma kind::f8f6f4, E4M3 x E4M3 -> F32, M=128 N=256
//                 K=32, both operands MN-major in shared memory (the shape and
//                 operand form of the tensor-core X-engine), issued back to
//                 back by one thread per SM into one TMEM accumulator
//   mma.sync s8   m16n8k32 int8 -> int32 on registers, four independent
//                 accumulators per warp (the int8 X-engine's instruction)
//   dp4a          four-way int8 dot products on registers, eight independent
//                 chains per thread (the CUDA-core X-engine's instruction)
//   fp32 FMA      paired fp32 FMAs (two multiply-adds an instruction, the fine
//                 filterbank's form), eight independent chains per thread
// The dp4a and FMA loops are unrolled so that loop overhead stays below 2 %.
//
// Every kernel runs one block per SM for a fixed number of iterations on
// values that stay in registers or shared memory; a sink store that never
// happens in practice keeps the work alive.  The rate is ops over the
// CUDA-event time of the launch (after one warm-up launch).
#include <cstdio>

#include "internal.cuh"

namespace corr {
namespace {

__device__ int g_probe_sink[4];

// ---------------------------------------------------------------- tcgen05 --
constexpr int kTcIters = 20000;                 // MMAs per SM
constexpr int kTcPlane = 8192;                  // one MN-major operand plane: 64 K-rows x 128 B
constexpr int kTcSmem = 3 * kTcPlane + 1024 + 64;
constexpr uint32_t kTcIdesc = (1u << 4) | (0u << 7) | (0u << 10) | (1u << 15) | (1u << 16) | ((256u >> 3) << 17) |
                              ((128u >> 4) << 24);

__device__ __forceinline__ uint64_t probe_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= uint64_t((saddr >> 4) & 0x3FFFu);
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
    d |= uint64_t(1) << 46;
    d |= uint64_t(2) << 61;   // 128-byte swizzle
    return d;
}

__global__ void __launch_bounds__(128, 1) probe_tc_kernel(long long wait_limit)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + 3 * kTcPlane);
    const uint32_t bar = sbase + 3 * kTcPlane + 16;
    for (int e = threadIdx.x; e < 3 * kTcPlane / 4; e += blockDim.x)
        reinterpret_cast<uint32_t *>(smem)[e] = 0x38383838u;   // E4M3 1.0: finite products
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
            static_cast<uint32_t>(__cvta_generic_to_shared(tmem_slot))));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    if (threadIdx.x == 0) {
        const uint64_t d = probe_desc(sbase, kTcPlane, 1024);
        const uint64_t dA = d, dB = d + uint64_t(kTcPlane >> 4);
        for (int k = 0; k < kTcIters; ++k) {
            const uint64_t off = uint64_t((k & 1) * (2048 >> 4));   // the two K halves of the planes
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(dA + off), "l"(dB + off), "r"(kTcIdesc), "r"(k));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                     : "memory");
        const long long t0 = clock64();
        uint32_t done = 0;
        while (!done && clock64() - t0 < wait_limit)
            asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
                         " selp.u32 %0, 1, 0, p;\n}\n"
                         : "=r"(done)
                         : "r"(bar)
                         : "memory");
        if (!done) atomicAdd(&g_probe_sink[3], 1);   // the MMAs did not finish in time
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

// ------------------------------------------------------------ register ones --
constexpr int kRegIters = 4096;

__global__ void __launch_bounds__(1024) probe_mma_s8_kernel(int seed)
{
    uint32_t a[4] = {uint32_t(seed), uint32_t(seed) * 3u, uint32_t(seed) * 5u, uint32_t(seed) * 7u};
    uint32_t b0 = uint32_t(threadIdx.x), b1 = uint32_t(threadIdx.x) * 11u;
    int d[4][4] = {};
#pragma unroll 1
    for (int k = 0; k < kRegIters; ++k) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                         "{%0,%1,%2,%3};\n"
                         : "+r"(d[c][0]), "+r"(d[c][1]), "+r"(d[c][2]), "+r"(d[c][3])
                         : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
    int x = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) x ^= d[c][0] ^ d[c][1] ^ d[c][2] ^ d[c][3];
    if (x == 0x7fedcba1) g_probe_sink[0] = x;
}

constexpr int kUnroll = 8;                      // loop bodies per iteration: loop overhead below 2 %

__global__ void __launch_bounds__(1024) probe_dp4a_kernel(int seed)
{
    int acc[8];
    const int a = seed * int(threadIdx.x + 1), b = seed ^ int(threadIdx.x);
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = c;
#pragma unroll 1
    for (int k = 0; k < kRegIters / kUnroll; ++k) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = __dp4a(a + c, b, acc[c]);
    }
    int x = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) x ^= acc[c];
    if (x == 0x7fedcba1) g_probe_sink[1] = x;
}

// paired fp32 FMAs (one instruction, two multiply-adds), as the filterbank uses
__global__ void __launch_bounds__(1024) probe_ffma_kernel(float seed)
{
    float2 acc[8];
    const float2 a = make_float2(seed * 0.999f, seed * 0.998f);
    const float2 b = make_float2(1.0f / (seed + float(threadIdx.x)), 0.5f / (seed + float(threadIdx.x)));
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = make_float2(float(c), float(c) + 0.5f);
#pragma unroll 1
    for (int k = 0; k < kRegIters / kUnroll; ++k) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = __ffma2_rn(acc[c], a, b);
    }
    float x = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) x += acc[c].x + acc[c].y;
    if (x == 1234.5f) g_probe_sink[2] = 1;
}

}  // namespace
}  // namespace corr

extern "C" int corr_probe_rate(int kind, double *ops_per_s, double *launch_ms, void *stream)
{
    using namespace corr;
    if (!ops_per_s || kind < CORR_PROBE_TC_FP8 || kind > CORR_PROBE_FFMA) return set_last_error(CORR_E_ARG);
    int dev = 0, sms = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev)) {
        cudaGetLastError();
        return set_last_error(CORR_E_CUDA);
    }
    if (kind == CORR_PROBE_TC_FP8 && !(major == 10 && minor == 3)) return set_last_error(CORR_E_UNSUPPORTED);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double ops = 0;
    auto launch = [&]() {
        switch (kind) {
        case CORR_PROBE_TC_FP8:
            probe_tc_kernel<<<sms, 128, kTcSmem, s>>>(1LL << 31);
            ops = double(sms) * kTcIters * 2.0 * 128 * 256 * 32;
            break;
        case CORR_PROBE_MMA_S8:
            probe_mma_s8_kernel<<<sms, 1024, 0, s>>>(3);
            ops = double(sms) * 32 * kRegIters * 4 * 2.0 * 16 * 8 * 32;
            break;
        case CORR_PROBE_DP4A:
            probe_dp4a_kernel<<<sms, 1024, 0, s>>>(3);
            ops = double(sms) * 1024 * kRegIters * 8 * 8.0;
            break;
        default:
            probe_ffma_kernel<<<sms, 1024, 0, s>>>(1.5f);
            ops = double(sms) * 1024 * kRegIters * 8 * 2 * 2.0;
            break;
        }
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    bool ok = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    if (ok) {
        launch();   // warm-up
        ok = cudaEventRecord(e0, s) == cudaSuccess;
        if (ok) launch();
        ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
             cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && cudaGetLastError() == cudaSuccess;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (!ok || ms <= 0.f) {
        cudaGetLastError();
        return set_last_error(CORR_E_CUDA);
    }
    int sink[4] = {0, 0, 0, 0};
    if (cudaMemcpyFromSymbol(sink, g_probe_sink, sizeof(sink)) != cudaSuccess) {
        cudaGetLastError();
        return set_last_error(CORR_E_CUDA);
    }
    if (kind == CORR_PROBE_TC_FP8 && sink[3] != 0) return set_last_error(CORR_E_TIMEOUT);
    *ops_per_s = ops / (double(ms) * 1e-3);
    if (launch_ms) *launch_ms = ms;
    return set_last_error(CORR_OK);
}
