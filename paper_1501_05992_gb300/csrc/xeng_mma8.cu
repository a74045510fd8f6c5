// X-engine, int8 tensor-core form (K2b): warp-level mma.sync m16n8k32
// s8 x s8 -> s32, exact.
//
// The complex product is embedded as a real dot product over K = 2T:
// row i of A is (r_i(0), m_i(0), r_i(1), m_i(1), ...), column j of B_re is the
// same vector of input j and column j of B_im is the twisted vector
// (-m_j(0), r_j(0), ...), so that A.B_re = Re V_ij and A.B_im = Im V_ij
// (V_ij = sum_t x_i conj(x_j), Eq. 3 integrated over time as in Section
// 3.4.2).  Tiles are 64 x 64 inputs per block (4 warps, 32 x 32 each), only
// lower-triangle tiles are launched, and operands come from the K-major
// staging written by the unpack kernel, through a 3-stage cp.async pipeline
// with an XOR-swizzled shared-memory layout so that ldmatrix is conflict-free.
//
// On sm_103 the tcgen05 int8 kind is not available (ptxas rejects
// tcgen05.mma kind::i8 for sm_103a), so this warp-level instruction is the
// int8 tensor path of this architecture.
#include "internal.cuh"

namespace corr {
namespace {

constexpr int T = kMmaTile;          // 64 inputs per tile side
constexpr int KT = kMmaKT;           // 64 samples per stage = 128 bytes per row
constexpr int kRowBytes = 2 * KT;    // 128
constexpr int kStages = 3;
constexpr int kThreads = 128;
constexpr int kTileBytes = T * kRowBytes;                     // 8 KB
constexpr int kStageBytes = 3 * kTileBytes;                   // A, B, Bt
constexpr int kSmemBytes = kStages * kStageBytes;             // 72 KB

__device__ __forceinline__ void cp_async16(uint32_t s, const void *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(g));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t addr, uint32_t &r0, uint32_t &r1,
                                            uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_s8(int (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                       uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// byte offset of 16-byte chunk `c` of row `r` in a 128-byte-row tile
__device__ __forceinline__ uint32_t swz(int r, int c) { return uint32_t(r * kRowBytes + ((c ^ (r & 7)) << 4)); }

__device__ __forceinline__ void tile_of(int b, int &bi, int &bj)
{
    int i = int((sqrtf(8.0f * float(b) + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= b) ++i;
    while (i * (i + 1) / 2 > b) --i;
    bi = i;
    bj = b - i * (i + 1) / 2;
}

template <bool kFresh>
__global__ void __launch_bounds__(kThreads)
xeng_mma8_kernel(const int8_t *__restrict__ X, const int8_t *__restrict__ Xt, int n, int n_pad,
                 int t_pad, int32_t *__restrict__ acc, int f0)
{
    extern __shared__ __align__(128) uint8_t smem[];
    int bi, bj;
    tile_of(blockIdx.x, bi, bj);
    const int fl = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wi = warp >> 1, wj = warp & 1;

    const size_t row_stride = size_t(t_pad) * 2;
    const int8_t *gA = X + (size_t(fl) * n_pad + bi * T) * row_stride;
    const int8_t *gB = X + (size_t(fl) * n_pad + bj * T) * row_stride;
    const int8_t *gBt = Xt + (size_t(fl) * n_pad + bj * T) * row_stride;
    const uint32_t s_base = static_cast<uint32_t>(__cvta_generic_to_shared(smem));

    auto load_stage = [&](int st, int kb) {
        const uint32_t sa = s_base + st * kStageBytes;
        const size_t koff = size_t(kb) * kRowBytes;
#pragma unroll
        for (int e = tid; e < T * 8; e += kThreads) {
            const int r = e >> 3, c = e & 7;
            const size_t go = r * row_stride + koff + c * 16;
            cp_async16(sa + swz(r, c), gA + go);
            cp_async16(sa + kTileBytes + swz(r, c), gB + go);
            cp_async16(sa + 2 * kTileBytes + swz(r, c), gBt + go);
        }
    };

    int re[2][4][4], im[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) re[a][b][c] = im[a][b][c] = 0;

    const int nk = t_pad / KT;
#pragma unroll
    for (int s = 0; s < kStages - 1; ++s) {
        if (s < nk) load_stage(s, s);
        cp_async_commit();
    }
    const int q = lane >> 3, r8 = lane & 7;
    for (int kb = 0; kb < nk; ++kb) {
        cp_async_wait<kStages - 2>();
        __syncthreads();
        if (kb + kStages - 1 < nk) load_stage((kb + kStages - 1) % kStages, kb + kStages - 1);
        cp_async_commit();
        const uint32_t sa = s_base + (kb % kStages) * kStageBytes;
        const uint32_t sb = sa + kTileBytes, sbt = sa + 2 * kTileBytes;
#pragma unroll
        for (int kk = 0; kk < KT / 16; ++kk) {      // 4 k32 steps (16 samples each)
            uint32_t a[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int row = wi * 32 + mt * 16 + (q & 1) * 8 + r8;
                const int chunk = 2 * kk + (q >> 1);
                ldmatrix_x4(sa + swz(row, chunk), a[mt][0], a[mt][1], a[mt][2], a[mt][3]);
            }
            uint32_t b[4][2], bt[4][2];
#pragma unroll
            for (int np = 0; np < 2; ++np) {
                const int row = wj * 32 + np * 16 + (q >> 1) * 8 + r8;
                const int chunk = 2 * kk + (q & 1);
                ldmatrix_x4(sb + swz(row, chunk), b[2 * np][0], b[2 * np][1], b[2 * np + 1][0],
                            b[2 * np + 1][1]);
                ldmatrix_x4(sbt + swz(row, chunk), bt[2 * np][0], bt[2 * np][1],
                            bt[2 * np + 1][0], bt[2 * np + 1][1]);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    mma_s8(re[mt][nt], a[mt], b[nt][0], b[nt][1]);
                    mma_s8(im[mt][nt], a[mt], bt[nt][0], bt[nt][1]);
                }
        }
    }
    cp_async_wait<0>();

    const long long P = n_pairs(n);
    int32_t *out = acc + (size_t)(f0 + fl) * P * 2;
    const int g = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = bi * T + wi * 32 + mt * 16 + g + 8 * h;
            if (i >= n) continue;
            const long long rowp = (long long)i * (i + 1) / 2;
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int j = bj * T + wj * 32 + nt * 8 + 2 * tig + e;
                    if (j > i) continue;
                    int2 *dst = reinterpret_cast<int2 *>(out + (rowp + j) * 2);
                    const int vr = re[mt][nt][2 * h + e], vi = im[mt][nt][2 * h + e];
                    if (kFresh) {
                        *dst = make_int2(vr, vi);
                    } else {
                        int2 v = *dst;
                        v.x += vr;
                        v.y += vi;
                        *dst = v;
                    }
                }
        }
}

}  // namespace

cudaError_t launch_xeng_mma8(const int8_t *X, const int8_t *Xt, int n, int n_pad, int fc,
                             int t_pad, int32_t *acc, int f0, bool fresh, cudaStream_t s)
{
    if (fc <= 0) return cudaSuccess;
    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncSetAttribute(xeng_mma8_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmemBytes);
        cudaFuncSetAttribute(xeng_mma8_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmemBytes);
        attr_done = true;
    }
    const int nb = n_pad / T;
    dim3 grid(nb * (nb + 1) / 2, fc);
    if (fresh)
        xeng_mma8_kernel<true><<<grid, kThreads, kSmemBytes, s>>>(X, Xt, n, n_pad, t_pad, acc, f0);
    else
        xeng_mma8_kernel<false><<<grid, kThreads, kSmemBytes, s>>>(X, Xt, n, n_pad, t_pad, acc, f0);
    return cudaGetLastError();
}

}  // namespace corr
