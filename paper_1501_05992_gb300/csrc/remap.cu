// Output remap (Appendix C, "GPU Output"), with optional further integration
// over adjacent channels and consecutive dumps (Section 3.4.3).
//
// The X-engine correlates the inputs in the order the PFBs deliver them
// (Appendix A: within each PFB's 64 inputs, position k carries input
// (k mod 4) * 16 + k div 4; Appendix B: the four PFBs' blocks follow each
// other) and writes the lower triangle over those positions.  The archived
// order is per station pair, natural input order, polarisation products
// innermost:
//
//     out[g][s1(s1+1)/2 + s2][p1][p2] = sum over dumps d and channels f of group g of
//                                       V_{2 s1 + p1, 2 s2 + p2}(f)
//
// with natural input a = 2 * station + pol.  V_AB with pos(A) >= pos(B) is a
// stored triangle element; otherwise it is the conjugate of the element
// (pos(B), pos(A)).  One thread writes the four polarisation products of one
// station pair (32 contiguous bytes); the inverse permutation lives in shared
// memory.  The kernel is bound by HBM (reads of
// the triangles, which the gather touches inside one channel's triangle at a
// time, and the coalesced writes).
#include "internal.cuh"

namespace corr {
namespace {

constexpr int kRemapThreads = 256;
constexpr int kRemapMaxDumps = 8;

struct RemapArgs {
    const int32_t *tri[kRemapMaxDumps];
    int n_dumps;
};

__device__ __forceinline__ int pfb_natural(int i)
{
    const int k = i & 63;
    return (i & ~63) + (k & 3) * 16 + (k >> 2);
}

__global__ void __launch_bounds__(kRemapThreads)
remap_kernel(RemapArgs args, int n, int n_chan, int f_avg, const int32_t *__restrict__ nat_of_pfb,
             int32_t *__restrict__ out)
{
    extern __shared__ int pos[];                    // pos[a]: PFB position of natural input a
    // every entry starts as a valid position, so a table that is not a
    // permutation gives wrong products but never an access out of bounds
    for (int a = threadIdx.x; a < n; a += blockDim.x) pos[a] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int a = nat_of_pfb ? nat_of_pfb[i] : pfb_natural(i);
        if (a >= 0 && a < n) pos[a] = i;
    }
    __syncthreads();
    const long long P = n_pairs(n);
    const int S = n / 2;
    const long long Q = n_pairs(S);
    const int g = blockIdx.y;
    // one thread per station pair: its four polarisation products are 32
    // contiguous output bytes
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < Q;
         q += (long long)gridDim.x * blockDim.x) {
        int s1 = int((sqrtf(8.0f * float(q) + 1.0f) - 1.0f) * 0.5f);
        while (n_pairs(s1 + 1) <= q) ++s1;
        while (n_pairs(s1) > q) --s1;
        const int s2 = int(q - n_pairs(s1));
        long long k[4];
        bool conj[4];
#pragma unroll
        for (int pp = 0; pp < 4; ++pp) {
            const int i = pos[2 * s1 + (pp >> 1)], j = pos[2 * s2 + (pp & 1)];
            conj[pp] = i < j;
            k[pp] = conj[pp] ? n_pairs(j) + i : n_pairs(i) + j;
        }
        int re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
        for (int d = 0; d < args.n_dumps; ++d) {
            for (int f = g * f_avg; f < (g + 1) * f_avg; ++f) {
                const int2 *tri = reinterpret_cast<const int2 *>(args.tri[d]) + (long long)f * P;
#pragma unroll
                for (int pp = 0; pp < 4; ++pp) {
                    const int2 v = __ldg(tri + k[pp]);
                    re[pp] += v.x;
                    im[pp] += v.y;
                }
            }
        }
        int4 *o = reinterpret_cast<int4 *>(out) + ((long long)g * Q + q) * 2;
        o[0] = make_int4(re[0], conj[0] ? -im[0] : im[0], re[1], conj[1] ? -im[1] : im[1]);
        o[1] = make_int4(re[2], conj[2] ? -im[2] : im[2], re[3], conj[3] ? -im[3] : im[3]);
    }
}

}  // namespace

cudaError_t launch_remap(const int32_t *const *tri, int n_dumps, int n, int n_chan, int f_avg,
                         const int32_t *nat_of_pfb, int32_t *out, cudaStream_t s)
{
    if (n_dumps < 1 || n_dumps > kRemapMaxDumps) return cudaErrorInvalidValue;
    RemapArgs args{};
    for (int d = 0; d < n_dumps; ++d) args.tri[d] = tri[d];
    args.n_dumps = n_dumps;
    const long long Q = n_pairs(n / 2);
    const long long want = (Q + kRemapThreads - 1) / kRemapThreads;
    const int bx = int(want < 4096 ? want : 4096);
    const dim3 grid(unsigned(bx), unsigned(n_chan / f_avg));
    remap_kernel<<<grid, kRemapThreads, size_t(n) * sizeof(int), s>>>(args, n, n_chan, f_avg, nat_of_pfb, out);
    return cudaGetLastError();
}

}  // namespace corr
