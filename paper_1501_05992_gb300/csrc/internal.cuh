// Internal declarations shared by the translation units of libcorr.so.
// Not part of the public ABI (that is include/corr.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "corr.h"

namespace corr {

// ----------------------------------------------------------------- sizes ---
constexpr int kDp4aTile = 64;          // CUDA-core X-engine tile (inputs per side)
constexpr int kDp4aKW = 32;            // 32-bit words (2 samples each) per K stage
constexpr int kMmaTile = 64;           // int8 mma.sync tile (inputs per side)
constexpr int kMmaKT = 64;             // samples per K stage of the mma.sync kernel
constexpr size_t kStageCap = size_t(1) << 30;  // unpacked-operand staging cap, bytes
constexpr int kHostChunk = 500;        // samples per host->device transfer chunk
constexpr int kHostBuffers = 3;        // device staging buffers of the host chunks
constexpr int kTcMaxSamples = 32768;   // tcgen05 path: samples per launch (FP32 sums < 2^24)
constexpr int kTcMaxArrays = 4;        // tcgen05 path: arrays correlated by one launch
constexpr size_t kAlign = 256;

__host__ __device__ inline long long n_pairs(long long n) { return n * (n + 1) / 2; }
inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
inline int div_up(int a, int b) { return (a + b - 1) / b; }

// Device status words written by kernels (index 0: error code, 1..3: detail).
struct DeviceStatus {
    int code;
    int where;
    int detail0;
    int detail1;
};

// Plan for the unpacked-operand paths (CUDA-core and mma.sync): the call's
// samples are processed in time chunks of t_chunk samples and channel chunks
// of f_chunk channels, each unpacked into the staging buffer then correlated.
struct StagePlan {
    int n_pad;        // inputs padded to the tile
    int t_chunk;      // samples per time chunk (even, multiple of the K stage)
    int f_chunk;      // channels per channel chunk
    size_t bytes;     // staging bytes needed
};

StagePlan plan_dp4a(int n_inputs, int n_chan, int t_max);
StagePlan plan_mma(int n_inputs, int n_chan, int t_max);

// ------------------------------------------------------------- launchers ---
// All launchers enqueue on `s` and return cudaGetLastError().

// Unpack channel chunk [f0, f0+fc) of samples [0, nt) of volt (uint8
// [*][n_chan][n] with row stride n_chan*n) into the dp4a operand planes:
// A[fc][tw_pad][n_pad] and W[fc][tw_pad][n_pad] (int8x4 words, two samples
// per word: (r0, m0, r1, m1) and (-m0, r0, -m1, r1)); zero beyond nt / n.
cudaError_t launch_unpack_words(const uint8_t *volt, int n_chan, int n, int f0, int fc,
                                int nt, int n_pad, int tw_pad, bool zero_invalid,
                                int32_t *A, int32_t *W, cudaStream_t s);

// Unpack into the K-major int8 layout out[fc][n_pad][t_pad][2] (real, imag),
// zero beyond nt / n; if out_tw is not NULL also the twisted plane (-m, r).
// Also used by corr_unpack with n_pad = n, t_pad = nt, out_tw = NULL.
cudaError_t launch_unpack_kmajor(const uint8_t *volt, int n_chan, int n, int f0, int fc,
                                 int nt, int n_pad, int t_pad, bool zero_invalid,
                                 int8_t *out, int8_t *out_tw, cudaStream_t s);

// Copy `rows` rows of n bytes (stride n in src) to a stride of ld >= n bytes
// in dst (the tensor-core path's 16-byte row alignment); bytes between rows
// are left as they are.
cudaError_t launch_pad_rows(const uint8_t *src, long long rows, int n, int ld, uint8_t *dst, cudaStream_t s);

// CUDA-core X-engine over a staged channel chunk; adds (or, if `fresh`,
// stores) into acc[f0 + fl][P][2].  tile: 32 or 64 inputs per side (n_pad a
// multiple of it).
cudaError_t launch_xeng_dp4a(const int32_t *A, const int32_t *W, int n, int n_pad, int fc,
                             int tw_pad, int32_t *acc, int f0, bool fresh, int tile, cudaStream_t s);

// int8 mma.sync X-engine over a staged K-major channel chunk (X and its
// twisted plane Xt, both [fc][n_pad][t_pad][2]).
cudaError_t launch_xeng_mma8(const int8_t *X, const int8_t *Xt, int n, int n_pad, int fc,
                             int t_pad, int32_t *acc, int f0, bool fresh, cudaStream_t s);

// tcgen05 FP8 X-engine straight from packed voltages (no staging).
bool tc_supported(int n_inputs, int device);
struct TcOptions {
    long long wait_limit = 0;   // bounded-wait limit in clock64 cycles (0: about 1 s)
    bool inject_stall = false;  // test hook: make the launch's first wait expire
};
// Work items of the tensor-core path: single 128 x 128 tile pairs, pair items
// (a diagonal tile and the tile left of it, sharing one conversion), or
// pairs only on launches of at least 64 stages.
enum class TcItems { kAuto = 0, kSingle = 1, kPairs = 2 };
struct TcArray {
    const uint8_t *volt;   // [nt][n_chan][ld] packed voltages (n used of each row of ld bytes)
    int32_t *acc;          // [n_chan][P][2] accumulators
    int n_chan, n, nt;
    bool zero_invalid, fresh;
    TcItems items = TcItems::kAuto;
    int ld = 0;            // row stride in bytes, a multiple of 16 (0: n)
    // incoherent beam of the same samples, added into beam[(beam_t0 + t) /
    // beam_avg][n_chan] (zeroed by the caller); NULL for none
    int32_t *beam = nullptr;
    int beam_avg = 1, beam_t0 = 0;
};
// Samples per padded copy for the tensor-core path when n % 16 != 0: the
// whole integration if it fits kTcPadCap bytes, else chunks of a multiple
// of 64 samples.
constexpr size_t kTcPadCap = size_t(4) << 30;
// One persistent launch over every (channel, tile pair) of up to
// kTcMaxArrays arrays (nt <= kTcMaxSamples each; arrays with nt == 0 skipped).
cudaError_t launch_xeng_tc_batch(const TcArray *arrays, int count, DeviceStatus *status,
                                 const TcOptions &opt, cudaStream_t s);

// Incoherent beam: out[k][f] = sum of |x|^2 over inputs and the n_avg samples
// of block k (n_time / n_avg blocks), int32.
cudaError_t launch_beam(const uint8_t *volt, int n_time, int n_chan, int n, int n_avg, bool zero_invalid,
                        int32_t *out, cudaStream_t s);

// Output remap of n_dumps PFB-order triangles tri[d] (int32 [n_chan][P][2])
// into station-pair order summed over dumps and f_avg channels:
// out int32 [n_chan / f_avg][S(S+1)/2][2][2][2], S = n / 2.  nat_of_pfb
// (device, n entries) or NULL for the Appendix A order.  n_dumps <= 8.
cudaError_t launch_remap(const int32_t *const *tri, int n_dumps, int n, int n_chan, int f_avg,
                         const int32_t *nat_of_pfb, int32_t *out, cudaStream_t s);

// Packet ingest of one bank (see corr_ingest_packets): zeroes seen and
// counters, scatters the good packets, marks unfilled slots invalid.
cudaError_t launch_ingest(const uint8_t *packets, long long n_packets, int bank, uint8_t *volt, void *seen,
                          int32_t *counters, cudaStream_t s);

// Fine polyphase filterbank (see corr_fine_pfb): x int8 [Q][N][S][2], window
// float [n_taps][128] (n_taps 1 or 12), outputs volt uint8 [M][Q*128][N]
// and/or spec float [M][Q*128][N][2] (either may be null), M = S/128 - n_taps + 1.
cudaError_t launch_fine_pfb(const int8_t *x, int n_coarse, int n_inputs, long long n_samples, const float *window,
                            int n_taps, float scale, uint8_t *volt, float *spec, cudaStream_t s);

// Record `status` as the calling thread's last error and return it.
int set_last_error(int status);

// Dump: vis = acc (or zeros if `fresh`), n_words int32 words.  *launches
// receives the number of kernels enqueued.
cudaError_t launch_dump(const int32_t *acc, int32_t *vis, size_t n_words, bool fresh,
                        cudaStream_t s, int *launches);

}  // namespace corr
