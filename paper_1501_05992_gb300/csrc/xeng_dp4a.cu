// X-engine, CUDA-core form (K2a): a register-tiled Hermitian rank-K update
// in exact int32 arithmetic on the SIMT integer pipes.
//
// This is the GB300 restatement of the paper's xGPU idea (Section 3.4.2): a
// thread block owns an m x n tile of baselines and integrates the products
// over time in registers, which raises the arithmetic intensity to
// 32mnI / (16(m+n)I + 64mn) (Eq. 4).  Here the tile is 64 x 64 (or 32 x 32)
// inputs per block, 8 x 4 per thread, and one dp4a instruction performs the four
// multiply-adds of two samples of one complex product:
//
//   a_i = (r_i(t), m_i(t), r_i(t+1), m_i(t+1))      the "words" plane
//   w_j = (-m_j(t), r_j(t), -m_j(t+1), r_j(t+1))    the "twisted" plane
//   dp4a(a_i, a_j) = sum over the 2 samples of  r_i r_j + m_i m_j  = Re
//   dp4a(a_i, w_j) = sum over the 2 samples of  m_i r_j - r_i m_j  = Im
//
// so Re/Im of V_ij = sum_t x_i conj(x_j) cost one dp4a each per two samples.
// Operands are staged through shared memory with cp.async double buffering.
// Only lower-triangle tiles (bj <= bi) are launched; a diagonal tile computes
// its full square and stores only j <= i.  Two tile shapes: 64 x 64 inputs
// (128 threads) and 32 x 32 (32 threads, less diagonal waste on small arrays).
#include "internal.cuh"

namespace corr {
namespace {

constexpr int KW = kDp4aKW;       // 32 words = 64 samples per stage
// tile T x T inputs per block; each thread owns 8 rows x 4 columns, so a
// block has (T/8) x (T/4) threads: 128 for T = 64, 32 for T = 32
template <int T>
__host__ __device__ constexpr int threads_for() { return (T / 8) * (T / 4); }

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void tile_of(int b, int &bi, int &bj)
{
    int i = int((sqrtf(8.0f * float(b) + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= b) ++i;
    while (i * (i + 1) / 2 > b) --i;
    bi = i;
    bj = b - i * (i + 1) / 2;
}

template <int T, bool kFresh>
__global__ void __launch_bounds__(threads_for<T>())
xeng_dp4a_kernel(const int32_t *__restrict__ A, const int32_t *__restrict__ W, int n,
                 int n_pad, int tw_pad, int32_t *__restrict__ acc, int f0)
{
    constexpr int kThreads = threads_for<T>();
    constexpr int kCols = T / 4;       // threads along j
    __shared__ __align__(16) int32_t sA[2][KW][T];
    __shared__ __align__(16) int32_t sB[2][KW][T];
    __shared__ __align__(16) int32_t sW[2][KW][T];

    int bi, bj;
    tile_of(blockIdx.x, bi, bj);
    const int fl = blockIdx.y;
    const int i_base = bi * T, j_base = bj * T;
    const int tid = threadIdx.x;
    const int tx = tid % kCols, ty = tid / kCols;

    const size_t plane = (size_t)fl * tw_pad * n_pad;
    const int32_t *gA = A + plane + i_base;
    const int32_t *gB = A + plane + j_base;
    const int32_t *gW = W + plane + j_base;

    auto load_stage = [&](int st, int k0) {
#pragma unroll
        for (int e = tid; e < KW * (T / 4); e += kThreads) {
            const int kk = e / (T / 4), c = e % (T / 4);
            const size_t go = (size_t)(k0 + kk) * n_pad + c * 4;
            cp_async16(&sA[st][kk][c * 4], gA + go);
            cp_async16(&sB[st][kk][c * 4], gB + go);
            cp_async16(&sW[st][kk][c * 4], gW + go);
        }
        cp_async_commit();
    };

    int re[8][4], im[8][4];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) re[r][c] = im[r][c] = 0;

    const int nk = tw_pad / KW;
    if (nk > 0) load_stage(0, 0);
    for (int kb = 0; kb < nk; ++kb) {
        if (kb + 1 < nk) {
            load_stage((kb + 1) & 1, (kb + 1) * KW);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int st = kb & 1;
#pragma unroll 4
        for (int k = 0; k < KW; ++k) {
            const int4 a0 = *reinterpret_cast<const int4 *>(&sA[st][k][ty * 8]);
            const int4 a1 = *reinterpret_cast<const int4 *>(&sA[st][k][ty * 8 + 4]);
            const int4 bb = *reinterpret_cast<const int4 *>(&sB[st][k][tx * 4]);
            const int4 ww = *reinterpret_cast<const int4 *>(&sW[st][k][tx * 4]);
            const int a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const int b[4] = {bb.x, bb.y, bb.z, bb.w};
            const int w[4] = {ww.x, ww.y, ww.z, ww.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    re[r][c] = __dp4a(a[r], b[c], re[r][c]);
                    im[r][c] = __dp4a(a[r], w[c], im[r][c]);
                }
        }
        __syncthreads();
    }

    const long long P = n_pairs(n);
    int32_t *out = acc + (size_t)(f0 + fl) * P * 2;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int i = i_base + ty * 8 + r;
        if (i >= n) continue;
        const long long row = (long long)i * (i + 1) / 2;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = j_base + tx * 4 + c;
            if (j > i) continue;
            int2 *dst = reinterpret_cast<int2 *>(out + (row + j) * 2);
            if (kFresh) {
                *dst = make_int2(re[r][c], im[r][c]);
            } else {
                int2 v = *dst;
                v.x += re[r][c];
                v.y += im[r][c];
                *dst = v;
            }
        }
    }
}

}  // namespace

template <int T>
cudaError_t launch_tile(const int32_t *A, const int32_t *W, int n, int n_pad, int fc, int tw_pad,
                        int32_t *acc, int f0, bool fresh, cudaStream_t s)
{
    const int nb = n_pad / T;
    dim3 grid(nb * (nb + 1) / 2, fc);
    if (fresh)
        xeng_dp4a_kernel<T, true><<<grid, threads_for<T>(), 0, s>>>(A, W, n, n_pad, tw_pad, acc, f0);
    else
        xeng_dp4a_kernel<T, false><<<grid, threads_for<T>(), 0, s>>>(A, W, n, n_pad, tw_pad, acc, f0);
    return cudaGetLastError();
}

cudaError_t launch_xeng_dp4a(const int32_t *A, const int32_t *W, int n, int n_pad, int fc,
                             int tw_pad, int32_t *acc, int f0, bool fresh, int tile, cudaStream_t s)
{
    if (fc <= 0) return cudaSuccess;
    if (n_pad % tile != 0) return cudaErrorInvalidValue;
    if (tile == 32) return launch_tile<32>(A, W, n, n_pad, fc, tw_pad, acc, f0, fresh, s);
    if (tile == 64) return launch_tile<64>(A, W, n, n_pad, fc, tw_pad, acc, f0, fresh, s);
    return cudaErrorInvalidValue;
}

}  // namespace corr
