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
// significant byte first.  Eight lanes take one packet (four packets per
// warp): lane j owns data words 8 j .. 8 j + 7, i.e. 32 sample bytes of one
// channel, loads the nine packet words that hold them (8-byte loads when the
// stream is 8-byte aligned, issued one packet ahead), realigns them (the data
// start at byte 6), XOR-reduces over the packet's lanes against the checksum,
// decodes the header from the words its neighbours hold, and stores its bytes
// with two 16-byte stores.  Sharing a warp among four packets divides the
// header decode and the reduction, which bound the one-packet-per-warp form.
// A slot is marked filled with a plain one-byte store (no value comes back, so
// no lane waits on it).  A second pass, one thread per (frame, group of four
// channels) reading the four PFBs' marks as one word, writes the slots no good
// packet filled with 0x88, the appendix's invalid code (CORR_ZERO_INVALID
// turns it into zeros), and counts them; the repeats are the good packets
// minus the distinct filled slots, added up in the same pass.
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

// The packet words lane j of a packet needs: W j .. W j + W + 1 (W = 64 / L).
template <int L, bool kAligned8>
struct PacketWords {
    static constexpr int W = 64 / L;
    uint32_t v[2 * (W / 2 + 1)];
    __device__ __forceinline__ void load(const uint32_t *w, int j)
    {
        if (kAligned8) {
            // words W j .. W j + W + 1 (word 0 of the packet is lane 0's first)
#pragma unroll
            for (int k = 0; k <= W / 2; ++k) {
                const uint2 u = __ldg(reinterpret_cast<const uint2 *>(w + W * j) + k);
                v[2 * k] = u.x;
                v[2 * k + 1] = u.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < W + 2; ++k) v[k] = __ldg(w + W * j + k);
        }
    }
    // packet word W j + k
    __device__ __forceinline__ uint32_t word(int k) const { return v[k]; }
};

template <int L, bool kAligned8>
__global__ void __launch_bounds__(kIngestThreads)
ingest_kernel(const uint32_t *__restrict__ pk, long long n_packets, int bank, uint8_t *__restrict__ volt,
              uint8_t *__restrict__ seen, int *__restrict__ counters)
{
    constexpr int P = 32 / L, W = 64 / L;
    const int lane = threadIdx.x & 31, sub = lane / L, j = lane % L;
    const long long warps = (long long)gridDim.x * (kIngestThreads / 32);
    __shared__ int block_counts[CORR_PKT_COUNTERS];
    if (threadIdx.x < CORR_PKT_COUNTERS) block_counts[threadIdx.x] = 0;
    __syncthreads();
    int mine[5] = {0, 0, 0, 0, 0};
    const long long step = warps * P;
    long long q0 = (blockIdx.x * (long long)(kIngestThreads / 32) + (threadIdx.x >> 5)) * P;
    PacketWords<L, kAligned8> cur;
    if (q0 < n_packets) cur.load(pk + min(q0 + sub, n_packets - 1) * kWords, j);
    // the loop runs for every lane of the warp (the shuffles below take all 32)
    for (; q0 < n_packets; q0 += step) {
        PacketWords<L, kAligned8> next;
        if (q0 + step < n_packets) next.load(pk + min(q0 + step + sub, n_packets - 1) * kWords, j);
        const long long q = q0 + sub;
        const bool valid = q < n_packets;
        // data word W j + k: packet bytes 6 + 4 (W j + k) .., from words W j + k + 1 and W j + k + 2
        uint32_t d[W];
        uint32_t x = 0;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            d[k] = __byte_perm(cur.word(k + 1), cur.word(k + 2), 0x5432);
            x ^= d[k];
        }
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) x ^= __shfl_xor_sync(0xFFFFFFFFu, x, o);
        const uint32_t w0 = __shfl_sync(0xFFFFFFFFu, cur.word(0), sub * L);
        const uint32_t w1 = __shfl_sync(0xFFFFFFFFu, cur.word(1), sub * L);
        const uint32_t w65 = __shfl_sync(0xFFFFFFFFu, cur.word(W + 1), sub * L + L - 1);
        if (valid) {
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
            if (j == 0) ++mine[code];
            if (code == CORR_PKT_GOOD) {
                const int cgroup = 32 * chan + 4 * mgt + grp;
                const long long slot = ((long long)frame * kGroups + cgroup) * 4 + pfb;
                if (j == 0) seen[slot] = 1;
                // data word l holds channel f2 = l / 16, inputs 64 pfb + 4 (l % 16) .. + 3
                const int l0 = W * j;
                uint4 *o = reinterpret_cast<uint4 *>(volt +
                                                     ((long long)frame * kChannels + 4 * cgroup + l0 / 16) * kInputs +
                                                     64 * pfb + 4 * (l0 % 16));
#pragma unroll
                for (int k = 0; k < W; k += 4) o[k / 4] = make_uint4(d[k], d[k + 1], d[k + 2], d[k + 3]);
            }
        }
        cur = next;
    }
    if ((lane % L) == 0)
        for (int c = 0; c < 5; ++c)
            if (mine[c]) atomicAdd(block_counts + c, mine[c]);
    __syncthreads();
    if (threadIdx.x < 5 && block_counts[threadIdx.x]) atomicAdd(counters + threadIdx.x, block_counts[threadIdx.x]);
}

// One thread per (frame, group of four channels): its four slots (one per PFB)
// are the four mark bytes of one word, and a slot nobody filled gets its four
// 64-byte runs of 0x88.
__global__ void __launch_bounds__(kIngestThreads)
ingest_missing_kernel(uint8_t *__restrict__ volt, const uint32_t *__restrict__ seen4, int *__restrict__ counters)
{
    int missing = 0;
    for (long long fg = blockIdx.x * (long long)kIngestThreads + threadIdx.x; fg < CORR_PKT_SLOTS / 4;
         fg += (long long)gridDim.x * kIngestThreads) {
        const uint32_t marks = seen4[fg];
        if ((marks & 0x000000FFu) && (marks & 0x0000FF00u) && (marks & 0x00FF0000u) && (marks & 0xFF000000u))
            continue;
        const long long frame = fg / kGroups, cgroup = fg % kGroups;   // fg = frame * kGroups + cgroup
        const uint4 inv = make_uint4(0x88888888u, 0x88888888u, 0x88888888u, 0x88888888u);
        for (int pfb = 0; pfb < 4; ++pfb) {
            if ((marks >> (8 * pfb)) & 0xFFu) continue;
#pragma unroll
            for (int f2 = 0; f2 < 4; ++f2) {
                uint4 *dst = reinterpret_cast<uint4 *>(volt + (frame * kChannels + 4 * cgroup + f2) * kInputs + 64 * pfb);
                dst[0] = inv;
                dst[1] = inv;
                dst[2] = inv;
                dst[3] = inv;
            }
            ++missing;
        }
    }
    __shared__ int block_missing;
    if (threadIdx.x == 0) block_missing = 0;
    __syncthreads();
    if (missing) atomicAdd(&block_missing, missing);
    __syncthreads();
    // repeats = good packets - distinct filled slots = GOOD - (SLOTS - MISSING):
    // every block adds its missing slots to both counters, and block 0 adds
    // GOOD - SLOTS (final: the ingest kernel ran before this one)
    if (threadIdx.x == 0) {
        int dup = block_missing;
        if (blockIdx.x == 0) dup += counters[CORR_PKT_GOOD] - CORR_PKT_SLOTS;
        if (block_missing) atomicAdd(counters + CORR_PKT_MISSING, block_missing);
        if (dup) atomicAdd(counters + CORR_PKT_DUPLICATE, dup);
    }
}

// The slot marks (one byte each, cleared four at a time) and the counters, in
// one launch.
__global__ void __launch_bounds__(kIngestThreads)
ingest_clear_kernel(uint32_t *__restrict__ seen4, int *__restrict__ counters)
{
    for (int e = blockIdx.x * kIngestThreads + threadIdx.x; e < CORR_PKT_SLOTS / 4; e += gridDim.x * kIngestThreads)
        seen4[e] = 0u;
    if (blockIdx.x == 0 && threadIdx.x < CORR_PKT_COUNTERS) counters[threadIdx.x] = 0;
}

}  // namespace

cudaError_t launch_ingest(const uint8_t *packets, long long n_packets, int bank, uint8_t *volt, void *seen,
                          int32_t *counters, cudaStream_t s)
{
    static_assert(CORR_PKT_SLOTS % 4 == 0, "four slots per mark word");
    ingest_clear_kernel<<<(CORR_PKT_SLOTS / 4 + kIngestThreads - 1) / kIngestThreads, kIngestThreads, 0, s>>>(
        static_cast<uint32_t *>(seen), counters);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (n_packets > 0) {
        constexpr int kL = 8;       // lanes per packet (8 measured faster than 4 and 16)
        const long long per_block = (kIngestThreads / 32) * (32 / kL);
        const long long blocks = (n_packets + per_block - 1) / per_block;
        // about two and a half passes per warp over a full bank: measured faster than
        // one pass (a block per 32 packets), five, or a persistent grid
        const unsigned grid = unsigned(blocks < 152 * 128 ? blocks : 152 * 128);
        const uint32_t *p32 = reinterpret_cast<const uint32_t *>(packets);
        if ((reinterpret_cast<uintptr_t>(packets) & 7) == 0)
            ingest_kernel<kL, true><<<grid, kIngestThreads, 0, s>>>(p32, n_packets, bank, volt,
                                                                     static_cast<uint8_t *>(seen), counters);
        else
            ingest_kernel<kL, false><<<grid, kIngestThreads, 0, s>>>(p32, n_packets, bank, volt,
                                                                      static_cast<uint8_t *>(seen), counters);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    ingest_missing_kernel<<<(CORR_PKT_SLOTS / 4 + kIngestThreads - 1) / kIngestThreads, kIngestThreads, 0, s>>>(
        volt, static_cast<const uint32_t *>(seen), counters);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace corr
