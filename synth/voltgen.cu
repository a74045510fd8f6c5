// GPU form of the seeded voltage generator in voltgen.py (same recipes, same
// bytes).  Input generation only: no correlator arithmetic lives here.  It
// exists so that workloads of tens of gigabytes can be created directly in
// device memory; any slice can be regenerated on the CPU with voltgen.py and
// compared byte for byte.
//
// Counter-based randomness: the SplitMix64 output function (Steele, Lea &
// Flood 2014) of key + (index + 1) * GAMMA.  Everything after the hash is
// integer fixed-point arithmetic identical to the numpy implementation.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kMix1 = 0xBF58476D1CE4E5B9ull;
constexpr uint64_t kMix2 = 0x94D049BB133111EBull;

__device__ __forceinline__ uint64_t hash_idx(uint64_t key, uint64_t idx)
{
    uint64_t z = key + (idx + 1ull) * kGamma;
    z = (z ^ (z >> 30)) * kMix1;
    z = (z ^ (z >> 27)) * kMix2;
    return z ^ (z >> 31);
}

__device__ __forceinline__ void ih4_pair(uint64_t h, int &a, int &b)
{
    int s0 = 0, s1 = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        s0 += int((h >> (8 * k)) & 0xFF);
        s1 += int((h >> (32 + 8 * k)) & 0xFF);
    }
    a = s0 - 510;
    b = s1 - 510;
}

__device__ __forceinline__ uint8_t quantise(int xr, int xi)
{
    int r = (xr + 2048) >> 12;
    int m = (xi + 2048) >> 12;
    r = r < -7 ? -7 : (r > 7 ? 7 : r);
    m = m < -7 ? -7 : (m > 7 ? 7 : m);
    return uint8_t(((r & 0xF) << 4) | (m & 0xF));
}

struct SrcKeys {
    uint64_t k[3];
};

__global__ void gauss3_kernel(uint8_t *__restrict__ out, int n_time, int n_chan, int n,
                              long long t0, int f0, int n_f, uint64_t key_noise, SrcKeys ks,
                              const int32_t *__restrict__ gains, int k_noise, int k_source)
{
    const long long total = (long long)n_time * n_f * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int ni = int(e % n);
        const long long rest = e / n;
        const int fl = int(rest % n_f);
        const long long tl = rest / n_f;
        const long long t = t0 + tl;
        const int f = f0 + fl;
        const uint64_t tf = uint64_t(t) * uint64_t(n_chan) + uint64_t(f);
        int nr, nim;
        ih4_pair(hash_idx(key_noise, tf * uint64_t(n) + uint64_t(ni)), nr, nim);
        int xr = (nr * k_noise) >> 8;
        int xi = (nim * k_noise) >> 8;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            int sr, si;
            ih4_pair(hash_idx(ks.k[s], tf), sr, si);
            sr = (sr * k_source) >> 8;
            si = (si * k_source) >> 8;
            const int32_t *g = gains + (((long long)s * n_chan + f) * n + ni) * 2;
            const int gr = g[0], gi = g[1];
            xr += (gr * sr - gi * si) >> 14;
            xi += (gr * si + gi * sr) >> 14;
        }
        out[e] = quantise(xr, xi);
    }
}

__global__ void uniform_tone_kernel(uint8_t *__restrict__ out, int n_time, int n_chan, int n,
                                    long long t0, int f0, int n_f, uint64_t key,
                                    const int32_t *__restrict__ tone)
{
    const long long total = (long long)n_time * n_f * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int ni = int(e % n);
        const long long rest = e / n;
        const int fl = int(rest % n_f);
        const long long tl = rest / n_f;
        const uint64_t idx = (uint64_t(t0 + tl) * uint64_t(n_chan) + uint64_t(f0 + fl)) * uint64_t(n) +
                             uint64_t(ni);
        const uint64_t h = hash_idx(key, idx);
        const int ur = int(((h & 0xFFFFFFFFull) * 15ull) >> 32) - 7;
        const int ui = int(((h >> 32) * 15ull) >> 32) - 7;
        const int32_t *tt = tone + (tl * n + ni) * 2;
        out[e] = quantise((ur << 12) + tt[0], (ui << 12) + tt[1]);
    }
}

int blocks_for(long long total)
{
    long long b = (total + 255) / 256;
    if (b < 1) b = 1;
    if (b > 152LL * 128) b = 152LL * 128;
    return int(b);
}

}  // namespace

extern "C" {

// out: device uint8 [n_time][n_f][n]; gains: device int32 [3][n_chan][n][2].
int vg_gauss3(uint8_t *out, int n_time, int n_chan, int n, long long t0, int f0, int n_f,
              uint64_t key_noise, uint64_t key_s0, uint64_t key_s1, uint64_t key_s2,
              const int32_t *gains, int k_noise, int k_source, void *stream)
{
    if (!out || !gains || n_time < 0 || n_chan < 1 || n < 1 || f0 < 0 || n_f < 0 ||
        f0 + n_f > n_chan)
        return -1;
    const long long total = (long long)n_time * n_f * n;
    if (total == 0) return 0;
    SrcKeys ks{{key_s0, key_s1, key_s2}};
    gauss3_kernel<<<blocks_for(total), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        out, n_time, n_chan, n, t0, f0, n_f, key_noise, ks, gains, k_noise, k_source);
    return cudaGetLastError() == cudaSuccess ? 0 : -6;
}

// out: device uint8 [n_time][n_f][n]; tone: device int32 [n_time][n][2] (Q12)
// for samples t0 .. t0 + n_time - 1.
int vg_uniform_tone(uint8_t *out, int n_time, int n_chan, int n, long long t0, int f0, int n_f,
                    uint64_t key, const int32_t *tone, void *stream)
{
    if (!out || !tone || n_time < 0 || n_chan < 1 || n < 1 || f0 < 0 || n_f < 0 ||
        f0 + n_f > n_chan)
        return -1;
    const long long total = (long long)n_time * n_f * n;
    if (total == 0) return 0;
    uniform_tone_kernel<<<blocks_for(total), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        out, n_time, n_chan, n, t0, f0, n_f, key, tone);
    return cudaGetLastError() == cudaSuccess ? 0 : -6;
}

}  // extern "C"
