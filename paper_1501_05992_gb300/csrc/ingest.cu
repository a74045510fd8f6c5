// Packet ingest: one 50 ms bank of PFB packets (Appendix A, "Data Format")
// into the assembled voltage block the X-engine reads (Appendix B: each
// packet's input order kept, the four PFBs concatenated; Appendix C "GPU
// Input": time, channel, input).
//
// Packet: 264 bytes = header word 0x0800, word two (sec_tick bit 0, pfb_id
// bits 4-5, mgt_id bits 6-8, mgt_bank bits 9-13), word three (mgt_frame bits
// 0-8, mgt_group bits 9-10, mgt_channel bits 11-15), 256 sample bytes (byte
// 64 f2 + k: fine channel 128 mgt_channel + 16 mgt_id + 4 mgt_group + f2,
// input 64 pfb_id + k), and the XOR of the 128 data words; 16-bit words most
// significant byte first.  One warp takes one packet: each lane realigns two
// 32-bit words of samples (they start at byte 6), the warp XOR-reduces them
// against the checksum, lane 0 decodes and checks the header and counters,
// and the lanes store the samples as four 64-byte runs.  Slots (frame, group
// of four channels, PFB) no good packet filled are then written with 0x88,
// the appendix's invalid code, which CORR_ZERO_INVALID turns into zeros.
// A slot is marked filled with a plain store (no value comes back, so the warp
// never waits on it), and the repeats are counted at the end as good packets
// minus distinct filled slots.
#include "internal.cuh"

namespace corr {
namespace {

constexpr int kFrames = CORR_PKT_FRAMES, kChannels = CORR_PKT_CHANNELS, kInputs = CORR_PKT_INPUTS;
constexpr int kGroups = kChannels / 4;
constexpr int kWords = CORR_PKT_BYTES / 4;     // 66 32-bit words per packet
constexpr int kIngestThreads = 256;

__device__ __forceinline__ unsigned be16(uint32_t w, int byte)   // big-endian 16-bit word at byte 0 or 2
{
    return ((w >> (8 * byte)) & 0xFFu) << 8 | ((w >> (8 * byte + 8)) & 0xFFu);
}

__global__ void __launch_bounds__(kIngestThreads)
ingest_kernel(const uint32_t *__restrict__ pk, long long n_packets, int bank, uint8_t *__restrict__ volt,
              uint32_t *__restrict__ seen, int *__restrict__ counters)
{
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (kIngestThreads / 32);
    // per-warp counts (lane 0), added to the block's and then once to the
    // global counters: one address hit by every packet would serialise
    __shared__ int block_counts[CORR_PKT_COUNTERS];
    if (threadIdx.x < CORR_PKT_COUNTERS) block_counts[threadIdx.x] = 0;
    __syncthreads();
    int mine[5] = {0, 0, 0, 0, 0};
    for (long long q = blockIdx.x * (long long)(kIngestThreads / 32) + (threadIdx.x >> 5); q < n_packets;
         q += warps) {
        const uint32_t *w = pk + q * kWords;
        // data word l: packet bytes 6 + 4l .. 9 + 4l, from 32-bit words 1 + l and 2 + l
        const uint32_t d0 = __byte_perm(__ldg(w + 1 + lane), __ldg(w + 2 + lane), 0x5432);
        const uint32_t d1 = __byte_perm(__ldg(w + 33 + lane), __ldg(w + 34 + lane), 0x5432);
        uint32_t x = d0 ^ d1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x ^= __shfl_xor_sync(0xFFFFFFFFu, x, o);
        const uint32_t w0 = __ldg(w), w1 = __ldg(w + 1), w65 = __ldg(w + 65);
        // even packet bytes are the words' high bytes: data bytes 0 and 2 of each group of four
        const unsigned xhi = (x ^ (x >> 16)) & 0xFFu, xlo = ((x >> 8) ^ (x >> 24)) & 0xFFu;
        const unsigned header = be16(w0, 0), word2 = be16(w0, 2), word3 = be16(w1, 0);
        const unsigned ck_hi = (w65 >> 16) & 0xFFu, ck_lo = (w65 >> 24) & 0xFFu;
        const int tick = int(word2 & 1u), pfb = int((word2 >> 4) & 3u), mgt = int((word2 >> 6) & 7u);
        const int bnk = int((word2 >> 9) & 31u);
        const int frame = int(word3 & 511u), grp = int((word3 >> 9) & 3u), chan = int((word3 >> 11) & 31u);
        int code = CORR_PKT_GOOD;
        if (header != 0x0800u) code = CORR_PKT_BAD_HEADER;
        else if (xhi != ck_hi || xlo != ck_lo) code = CORR_PKT_BAD_CHECKSUM;
        else if (bnk != bank || chan >= 24 || frame >= kFrames ||
                 (tick && (bnk | chan | grp | frame) != 0))
            code = CORR_PKT_BAD_FIELD;
        if (code != CORR_PKT_GOOD) {
            ++mine[code];
            continue;
        }
        const int cgroup = 32 * chan + 4 * mgt + grp;
        const long long slot = ((long long)frame * kGroups + cgroup) * 4 + pfb;
        if (lane == 0) seen[slot] = 1u;
        ++mine[CORR_PKT_GOOD];
        // data word l holds channel f2 = l / 16, inputs 64 pfb + 4 (l % 16) .. + 3
        const long long base = ((long long)frame * kChannels + 4 * cgroup) * kInputs + 64 * pfb + 4 * (lane & 15);
        uint32_t *o = reinterpret_cast<uint32_t *>(volt);
        o[(base + (long long)(lane >> 4) * kInputs) >> 2] = d0;
        o[(base + (long long)(2 + (lane >> 4)) * kInputs) >> 2] = d1;
    }
    if (lane == 0)
        for (int c = 0; c < 5; ++c)
            if (mine[c]) atomicAdd(block_counts + c, mine[c]);
    __syncthreads();
    if (threadIdx.x < 5 && block_counts[threadIdx.x]) atomicAdd(counters + threadIdx.x, block_counts[threadIdx.x]);
}

// One thread per (slot, channel f2): a slot nobody filled gets 64 bytes of 0x88.
__global__ void __launch_bounds__(kIngestThreads)
ingest_missing_kernel(uint8_t *__restrict__ volt, const uint32_t *__restrict__ seen, int *__restrict__ counters)
{
    const long long n = (long long)CORR_PKT_SLOTS * 4;
    int missing = 0;
    for (long long e = blockIdx.x * (long long)kIngestThreads + threadIdx.x; e < n;
         e += (long long)gridDim.x * kIngestThreads) {
        const long long slot = e >> 2;
        if (seen[slot]) continue;
        const int f2 = int(e & 3);
        const int pfb = int(slot & 3);
        const long long fg = slot >> 2;                 // frame * kGroups + cgroup
        const long long frame = fg / kGroups, cgroup = fg % kGroups;
        uint4 *dst = reinterpret_cast<uint4 *>(volt + (frame * kChannels + 4 * cgroup + f2) * kInputs + 64 * pfb);
        const uint4 inv = make_uint4(0x88888888u, 0x88888888u, 0x88888888u, 0x88888888u);
        dst[0] = inv;
        dst[1] = inv;
        dst[2] = inv;
        dst[3] = inv;
        if (f2 == 0) ++missing;
    }
    __shared__ int block_missing;
    if (threadIdx.x == 0) block_missing = 0;
    __syncthreads();
    if (missing) atomicAdd(&block_missing, missing);
    __syncthreads();
    if (threadIdx.x == 0 && block_missing) atomicAdd(counters + CORR_PKT_MISSING, block_missing);
}

// Repeated packets: every good packet fills one slot, so the repeats are the
// good packets beyond the distinct slots filled (all slots but the missing).
__global__ void ingest_repeats_kernel(int *__restrict__ counters)
{
    counters[CORR_PKT_DUPLICATE] =
        counters[CORR_PKT_GOOD] - (CORR_PKT_SLOTS - counters[CORR_PKT_MISSING]);
}

}  // namespace

cudaError_t launch_ingest(const uint8_t *packets, long long n_packets, int bank, uint8_t *volt, void *seen,
                          int32_t *counters, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(seen, 0, size_t(CORR_PKT_SEEN_BYTES), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, sizeof(int32_t) * CORR_PKT_COUNTERS, s);
    if (e != cudaSuccess) return e;
    if (n_packets > 0) {
        const long long blocks = (n_packets + kIngestThreads / 32 - 1) / (kIngestThreads / 32);
        ingest_kernel<<<unsigned(blocks < 152 * 64 ? blocks : 152 * 64), kIngestThreads, 0, s>>>(
            reinterpret_cast<const uint32_t *>(packets), n_packets, bank, volt, static_cast<uint32_t *>(seen),
            counters);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    ingest_missing_kernel<<<152 * 32, kIngestThreads, 0, s>>>(volt, static_cast<const uint32_t *>(seen), counters);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ingest_repeats_kernel<<<1, 1, 0, s>>>(counters);
    return cudaGetLastError();
}

}  // namespace corr
