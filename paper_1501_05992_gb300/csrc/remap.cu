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
// (pos(B), pos(A)).  One thread owns one station pair: it finds the pair's
// four triangle elements once and then gathers them from every (dump,
// channel) of each channel group its block visits, four (group, dump,
// channel) triples at a time (16 loads in flight), writing the four
// polarisation products of a group (32 contiguous bytes) after its last
// triple; the inverse permutation lives in shared memory, built once per
// block.  The kernel is bound by HBM (reads of the triangles, which the gather
// touches inside one channel's triangle at a time, and the coalesced writes).
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
    const int n_groups = n_chan / f_avg, n_comb = args.n_dumps * f_avg;
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
        // the (channel group, dump, channel) triples of this thread's station pair,
        // groups blockIdx.y + j gridDim.y, taken four at a time (16 loads in flight)
        const int n_j = (n_groups - int(blockIdx.y) + int(gridDim.y) - 1) / int(gridDim.y);
        const int n_e = n_j * n_comb;
        int re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
        for (int e0 = 0; e0 < n_e; e0 += 4) {
            int2 v[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u < n_e ? e0 + u : e0;   // past the end: repeat, not added
                const int j = e / n_comb, c = e - j * n_comb;
                const int g = int(blockIdx.y) + j * int(gridDim.y);
                const int d = c / f_avg, f = g * f_avg + (c - d * f_avg);
                // select the dump's pointer without indexing the parameter array
                const int32_t *base = args.tri[0];
#pragma unroll
                for (int x = 1; x < kRemapMaxDumps; ++x)
                    if (x == d) base = args.tri[x];
                const int2 *tri = reinterpret_cast<const int2 *>(base) + (long long)f * P;
#pragma unroll
                for (int pp = 0; pp < 4; ++pp) v[u][pp] = __ldg(tri + k[pp]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u;
                if (e >= n_e) break;
#pragma unroll
                for (int pp = 0; pp < 4; ++pp) {
                    re[pp] += v[u][pp].x;
                    im[pp] += v[u][pp].y;
                }
                const int j = e / n_comb;
                if (e - j * n_comb == n_comb - 1) {
                    // the group's last triple: write its four products and start the next
                    const int g = int(blockIdx.y) + j * int(gridDim.y);
                    int4 *o = reinterpret_cast<int4 *>(out) + ((long long)g * Q + q) * 2;
                    o[0] = make_int4(re[0], conj[0] ? -im[0] : im[0], re[1], conj[1] ? -im[1] : im[1]);
                    o[1] = make_int4(re[2], conj[2] ? -im[2] : im[2], re[3], conj[3] ? -im[3] : im[3]);
#pragma unroll
                    for (int pp = 0; pp < 4; ++pp) re[pp] = im[pp] = 0;
                }
            }
        }
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
    // a block builds the permutation table once and visits several channel
    // groups: about 1600 blocks at 256 inputs
    const int groups = n_chan / f_avg;
    const int by = groups < 48 ? groups : 48;
    const dim3 grid{unsigned(bx), unsigned(by)};
    remap_kernel<<<grid, kRemapThreads, size_t(n) * sizeof(int), s>>>(args, n, n_chan, f_avg, nat_of_pfb, out);
    return cudaGetLastError();
}

}  // namespace corr
