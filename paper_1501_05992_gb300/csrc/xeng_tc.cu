// X-engine, tcgen05 FP8 tensor-core form (K2c), fused with the unpack.
//
// What it computes is Eq. 3 (Section 2) integrated over time (Section 3.4.2):
// V_ij(f) = sum_t x_i(t,f) conj(x_j(t,f)) for j <= i, straight from the
// packed 4+4-bit voltages volt[t][f][n] (Appendix A, Appendix C "GPU Input"),
// into the packed lower triangle of Appendix C "GPU Output".  The paper's GPU
// kernel (xGPU) tiles baselines per thread block and integrates in registers
// (Section 3.4.2, Eq. 4); here a baseline tile is a 128 x 128 block of inputs
// integrated in tensor memory (TMEM) by tcgen05.mma.
//
// Encoding (exact): each 4-bit two's-complement component v in [-8, 7] is
// coded as u = v + 8 in [0, 15], and the E4M3 byte with bit pattern u
// (0x00..0x0F) has the value u * 2^-9: codes 1..7 are subnormals, 8..15 the
// first normal binade, so the byte map is one XOR with 0x08 per nibble.  The
// tensor core then computes, per sample, products u_i u_j * 2^-18, exact in
// FP32, and FP32 accumulation stays exact while |sum| < 2^24 (measured on
// sm_103a; the host splits calls at kTcMaxSamples so the bound always holds).
// With ur, um the codes of the real and imaginary parts:
//
//   P_re = sum(ur_i ur_j + um_i um_j),  P_im = sum(um_i ur_j - ur_i um_j)
//   Re V_ij = P_re - 8 (E_i + E_j) + 128 T,   Im V_ij = P_im - 8 D_i + 8 D_j
//
// with E_k = sum(ur_k + um_k), D_k = sum(um_k - ur_k) over the T processed
// samples (samples past the end of the block are zero bytes, i.e. u = 8, and
// cancel exactly).
//
// Complex -> real: for the tile pair (I, J), I >= J, the MMA's A operand (the
// 128 TMEM lanes) is the J tile and its B operand (the TMEM columns) the I
// tile.  With planes R (ur), M (um), nM (-um), two MMAs per 32 samples, each
// M=128 x N=256 x K=32, fill D = [Re | Im]:
//   D += R_J . [R_I ; nM_I]^T   ->  [ sum ur_j ur_i | -sum ur_j um_i ]
//   D += M_J . [M_I ; R_I ]^T   ->  [ sum um_j um_i |  sum um_j ur_i ]
// i.e. D[a][b] = sum x_a conj(x_b) for input a of J and b of I, and V_ij =
// conj(D[a][b]).  Operands are MN-major (inputs contiguous, the natural
// [t][n] order of the voltages), 128-byte swizzled, so no transpose is ever
// needed.  Lanes on the J side make the epilogue's stores coalesced: a TMEM
// column read gives 32 lanes = 32 consecutive elements of one packed row.
//
// Work items: per channel, a diagonal tile (I, I) and the tile left of it
// (I, I - 1) form one "pair" item, since both multiply by the I tile's planes
// as B: the pair converts the two tiles once and issues both MMA chains, into
// the two TMEM accumulators.  The other tiles (J <= I - 2) are single items,
// and the first diagonal (0, 0) is a single item too (for 256 inputs: one pair
// and one diagonal item per channel, where single items would make three).
// Launches shorter than kPairMinStages stages use single items only.
//
// Pipeline (persistent, one CTA per SM, work item = (channel, I tile, J tile)):
//   warp 0     TMA producer: packed bytes [64 samples][128 inputs] per tile,
//              with L2 prefetch of the tiles kPrefetchStages stages ahead
//              (across item boundaries: an item's last stages prefetch the
//              CTA's next item's first)
//   warp 1     TMEM allocator and single-thread MMA issuer
//   warps 2-16, 22  converters: packed bytes -> E4M3 planes (+ per-input
//              sums), as two teams of 8 warps that take alternate 64-sample
//              stages (a warp's barrier waits and arrivals cost about as much as
//              its conversion work, so a team owning whole stages halves that
//              cost); warp 17 is left idle so that the MMA warp's scheduler
//              (warps 1, 5, 9, ... share one) serves one converter warp fewer
//   warps 18-21 epilogue: TMEM -> int32, corrections, packed-triangle store
//              (fp32 on exact integers; each store instruction writes 32
//              consecutive elements of one packed row)
//   warps 23-26 (launches that also form the incoherent beam only): the
//              total power of each tile's inputs per sample, read from the
//              packed bytes in shared memory and added into the beam (warps
//              23-24 the B tile's rows, 25-26 the A tile's)
// TMEM holds two accumulators (2 x 256 columns).  A single item takes the
// next one in turn, so its epilogue overlaps the main loop of the next item; a
// pair item takes both, its diagonal part in the one that is released first.
// Every wait is bounded: on
// a timeout the kernel records CORR_E_TIMEOUT, drains its own copies and MMAs,
// frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.cuh"

namespace corr {
namespace {

constexpr int kTile = 128;                    // inputs per tile side
constexpr int kMaxArrays = kTcMaxArrays;      // arrays correlated by one launch
constexpr int kTc = 64;                       // samples per pipeline stage
constexpr int kPackedStages = 6;
constexpr int kPrefetchStages = 12;           // L2 prefetch distance of the packed loads
constexpr int kPlaneStages = 3;
constexpr int kPlaneBytes = kTc * 128;        // one E4M3 plane: 64 rows x 128 B = 8 KB
constexpr int kPackedTileBytes = kTc * kTile; // 8 KB
constexpr int kPackedStageBytes = 2 * kPackedTileBytes;
// plane stage layout: R_A | M_A | M_B | R_B | nM_B (A: the tile of the TMEM
// rows, the output's column inputs; B: the tile of the TMEM columns, the
// output's row inputs)
constexpr int kOffRA = 0, kOffMA = kPlaneBytes, kOffMB = 2 * kPlaneBytes, kOffRB = 3 * kPlaneBytes,
              kOffNMB = 4 * kPlaneBytes;
constexpr int kPlaneStageBytes = 5 * kPlaneBytes;  // 40 KB
constexpr int kConvWarps = 16, kEpiWarps = 4;
constexpr int kTeams = 2, kTeamWarps = kConvWarps / kTeams;   // converter teams own alternate stages
// A team waits on the packed slot of stage g with the parity of g's use of the
// slot.  That is unambiguous only if the slot's previous use (g - kPackedStages)
// was the same team's, already consumed: with a slot count that is not a
// multiple of the team count the previous use is the other team's, its copy
// may still be in flight, and the parity of use g would match the completed
// use g - 2 kPackedStages.  (Plane slots are waited on by the in-order MMA
// issuer, and their "empty" waits are ordered by it, so any count works.)
static_assert(kPackedStages % kTeams == 0, "packed slots must be team-exclusive");
constexpr int kThreads = (2 + kConvWarps + kEpiWarps + 1) * 32;   // 736: warp 22 converts, warp 17 idles
constexpr int kFirstConvWarp = 2, kFirstEpiWarp = 2 + kConvWarps;
// With the incoherent beam, warps 23-26 form it from the packed bytes in
// shared memory (32 rows of one tile of each stage each); at 72 registers a
// thread the launch's 864 threads fit the register file.
constexpr int kBeamWarps = 4, kFirstBeamWarp = kThreads / 32;
constexpr int kThreadsBeam = kThreads + kBeamWarps * 32;   // 864
constexpr int kTmemCols = 512;               // 2 accumulator slots x (128 Re + 128 Im)
// A pair item needs both TMEM accumulators free before its first MMA, so the
// previous item's epilogue is exposed once per pair.  On short launches that
// costs more than the shared conversion saves, so pairs are used only from
// this many stages on (measured crossover 32 to 64 stages for 256 and 512
// inputs, whether the epilogue stores or adds into the output).
constexpr int kPairMinStages = 64;
constexpr long long kDefaultWaitLimit = 1LL << 31;  // clock64 cycles (about 1 s)

// shared-memory map (offsets from a 1024-aligned base)
constexpr int kSmPacked = 0;
constexpr int kSmPlanes = kSmPacked + kPackedStages * kPackedStageBytes;          // 96 KB
constexpr int kSmSums = kSmPlanes + kPlaneStages * kPlaneStageBytes;              // +120 KB
constexpr int kSumsBytes = 2 * 2 * 2 * kTile * 4;                                 // [buf][tile][r/m][slot]
constexpr int kSmBars = kSmSums + kSumsBytes;
constexpr int kNumBars = 2 * kPackedStages + 2 * kPlaneStages + 4 + 4 + 2;
constexpr int kSmMisc = kSmBars + kNumBars * 8;
constexpr int kSmemBytes = kSmMisc + 64 + 1024;                                   // + alignment slack

// instruction descriptor: kind::f8f6f4, E4M3 x E4M3 -> F32, both MN-major, M=128, N=256
constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | (1u << 15) | (1u << 16) |
                            ((256u >> 3) << 17) | ((128u >> 4) << 24);

// One array of a launch.  The work items of array a are numbered
// item_begin .. item_begin + n_chan * per_chan - 1; the host orders
// the arrays by decreasing n_stages so that a CTA's last items are its
// shortest (a static longest-first schedule).
struct ArrayParams {
    int32_t *acc;
    int n, n_chan, nt, n_tiles, per_chan, n_stages, item_begin;
    int fresh;
    int pairs;      // pair items in use (else one item per tile pair)
    int rot_step;   // item rotation per stride round (see decode_item)
    int32_t *beam;  // incoherent beam [.][beam_ld], added to (NULL: none)
    int beam_ld;    // channels of a beam row
    int beam_avg, beam_t0;   // samples per beam value; the launch's first sample
};

struct Params {
    ArrayParams a[kMaxArrays];
    int n_arrays, n_items;
    DeviceStatus *status;
    long long wait_limit;   // bounded-wait limit, clock64 cycles
    int inject_stall;       // test hook: the epilogue first waits on a barrier nobody arrives on
};

struct Tmaps {
    CUtensorMap m[kMaxArrays];
};

// ------------------------------------------------------------ PTX helpers --
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// As mbar_try, but a thread whose phase is not complete may be suspended for
// up to 1 ms (it resumes as soon as the phase completes), so bounded waits
// poll rarely instead of spinning.
__device__ __forceinline__ bool mbar_try_sleep(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity), "n"(1000000)
        : "memory");
    return done != 0;
}

// Bounded wait.  Returns false on timeout or if another role aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort,
                                          DeviceStatus *status, int where, long long limit)
{
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_sleep(bar, parity)) return true;
        if (*abort) return false;
        if (clock64() - t0 > limit) {
            *abort = 1;
            if (atomicCAS(&status->code, 0, CORR_E_TIMEOUT) == 0) {
                status->where = where;
                status->detail0 = int(blockIdx.x);
            }
            return false;
        }
    }
}

// Warp-wide bounded wait: lane 0 polls (with an optional back-off), then every
// lane confirms once, so each lane gets the barrier's acquire ordering while
// only one lane keeps hitting shared memory.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int *abort,
                                          DeviceStatus *status, int where, int lane, long long limit,
                                          unsigned sleep_ns = 0)
{
    int ok = 1;
    if (lane == 0) {
        if (!mbar_try(bar, parity)) {
            const long long t0 = clock64();
            while (true) {
                if (mbar_try(bar, parity)) break;
                if (*abort) {
                    ok = 0;
                    break;
                }
                if (clock64() - t0 > limit) {
                    *abort = 1;
                    if (atomicCAS(&status->code, 0, CORR_E_TIMEOUT) == 0) {
                        status->where = where;
                        status->detail0 = int(blockIdx.x);
                    }
                    ok = 0;
                    break;
                }
                if (sleep_ns) __nanosleep(sleep_ns);
            }
        }
    }
    ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
    if (!ok) return false;
    return mbar_try(bar, parity);        // completed: returns at once, with acquire
}

// index of input n (0..127) in a row of per-input sums: [n % 16][n / 16], so
// that the eight lanes adding sums of the same offset within their 16-input
// chunk hit eight consecutive words (no bank conflicts)
__device__ __forceinline__ int sum_slot(int n) { return (n & 15) * 8 + (n >> 4); }

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap *map, int x, int y, int z)
{
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z)
                 : "memory");
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= uint64_t((saddr >> 4) & 0x3FFFu);
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
    d |= uint64_t(1) << 46;                     // descriptor version
    d |= uint64_t(2) << 61;                     // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void mma_f8(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accum)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void named_sync(int id, int threads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Work items of one channel, for n_tiles tiles of 128 inputs (tile pair (I, J)
// with I >= J: output rows in tile I, columns in tile J): the diagonal item
// (0, 0), then for each I >= 1 a pair item covering (I, I) and (I, I - 1) (both
// multiply by the I tile's planes as the B operand, so one conversion feeds
// both, into two accumulators) and the off-diagonal items (I, J) for
// J <= I - 2.  n_tiles (n_tiles + 1) / 2 - (n_tiles - 1) items per channel.
enum ItemKind { kDiagItem = 0, kOffItem = 1, kPairItem = 2 };

__host__ __device__ __forceinline__ int items_per_channel(int n_tiles, bool pairs)
{
    return n_tiles * (n_tiles + 1) / 2 - (pairs ? n_tiles - 1 : 0);
}

__host__ __device__ __forceinline__ void item_tiles(int k, int n_tiles, bool pairs, int &I, int &J, int &kind)
{
    if (!pairs) {
        // one item per tile pair, numbered row by row of the tile triangle
        int i = int((sqrtf(8.0f * float(k) + 1.0f) - 1.0f) * 0.5f);
        while ((i + 1) * (i + 2) / 2 <= k) ++i;
        while (i * (i + 1) / 2 > k) --i;
        I = i;
        J = k - i * (i + 1) / 2;
        kind = I == J ? kDiagItem : kOffItem;
        return;
    }
    if (k == 0) {
        I = J = 0;
        kind = kDiagItem;
        return;
    }
    --k;
    for (I = 1; I + 1 < n_tiles && k >= I; ++I) k -= I;   // row I holds I items
    if (k == 0) {
        J = I - 1;
        kind = kPairItem;
    } else {
        J = k - 1;
        kind = kOffItem;
    }
}

struct Item {
    int a, f, I, J, kind;
    bool diag;      // the producer and the converters see a pair item as the off-diagonal (I, I - 1)
};

__device__ __forceinline__ Item decode_item(const Params &p, int item)
{
    Item it;
    it.a = 0;
    while (it.a + 1 < p.n_arrays && item >= p.a[it.a + 1].item_begin) ++it.a;
    const ArrayParams &A = p.a[it.a];
    const int local = item - A.item_begin;
    it.f = local / A.per_chan;
    // The CTAs take items with a stride of g = gridDim.x, so with c items per
    // channel a CTA would meet the same item kind every round whenever g is a
    // multiple of c (e.g. 2 items per channel on 152 CTAs).  In that case the
    // host sets rot_step = 1: a channel's items rotate by one per stride round
    // of its first item, and each CTA steps through the kinds in turn.  (When
    // c does not divide g the stride itself moves a CTA through the kinds.)
    // A rotation within every channel is a bijection, so all roles of the CTA
    // agree on it.
    const int k = local - it.f * A.per_chan;
    const int round = (A.item_begin + it.f * A.per_chan) / int(gridDim.x);
    item_tiles(A.rot_step ? (k + round) % A.per_chan : k, A.n_tiles, A.pairs != 0, it.I, it.J, it.kind);
    it.diag = it.kind == kDiagItem;
    return it;
}

// 256 (r^2 + m^2) summed over the 4 packed samples of w, plus acc: the high
// nibble with the low one cleared is the signed byte 16 r, the low nibble
// moved up the signed byte 16 m (Appendix A: two's complement, real high).
// With zero_invalid, samples with a nibble of 8 count as zero.
__device__ __forceinline__ int power256(uint32_t w, bool zero_invalid, int acc)
{
    uint32_t hr = w & 0xF0F0F0F0u, hm = (w << 4) & 0xF0F0F0F0u;
    if (zero_invalid) {
        const uint32_t bad = __vcmpeq4(hr, 0x80808080u) | __vcmpeq4(hm, 0x80808080u);
        hr &= ~bad;
        hm &= ~bad;
    }
    return __dp4a(int(hm), int(hm), __dp4a(int(hr), int(hr), acc));
}

// 4 packed bytes (r << 4 | m) -> E4M3 codes u = nibble ^ 8 (value u * 2^-9).
__device__ __forceinline__ void codes(uint32_t w, bool zero_invalid, uint32_t &R, uint32_t &M)
{
    R = ((w >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
    M = (w & 0x0F0F0F0Fu) ^ 0x08080808u;
    if (zero_invalid) {
        // a nibble code of 8 (value -8) has u == 0: such samples become 0 + 0i (u = 8, 8)
        const uint32_t nzR = (R + 0x7F7F7F7Fu) & 0x80808080u;   // bit 7 set where u != 0
        const uint32_t nzM = (M + 0x7F7F7F7Fu) & 0x80808080u;
        const uint32_t bad = (~(nzR & nzM)) & 0x80808080u;      // bit 7 set where invalid
        const uint32_t mask = (bad >> 7) * 0xFFu;
        R = (R & ~mask) | (0x08080808u & mask);
        M = (M & ~mask) | (0x08080808u & mask);
    }
}

// kBeam: the converters also add the incoherent beam (Section 3.4: the total
// power of all inputs per channel and sample) of the arrays that ask for it.
template <bool kZeroInvalid, bool kBeam>
__global__ void __launch_bounds__(kBeam ? kThreadsBeam : kThreads, 1)
xeng_tc_kernel(const __grid_constant__ Tmaps tmaps, const __grid_constant__ Params p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    int *sums = reinterpret_cast<int *>(smem + kSmSums);
    const uint32_t bars = sbase + kSmBars;
    auto bar_packed_full = [&](int s) { return bars + 8u * s; };
    auto bar_packed_empty = [&](int s) { return bars + 8u * (kPackedStages + s); };
    auto bar_plane_full = [&](int s) { return bars + 8u * (2 * kPackedStages + s); };
    auto bar_plane_empty = [&](int s) { return bars + 8u * (2 * kPackedStages + kPlaneStages + s); };
    auto bar_acc_full = [&](int b) { return bars + 8u * (2 * kPackedStages + 2 * kPlaneStages + b); };
    auto bar_acc_empty = [&](int b) { return bars + 8u * (2 * kPackedStages + 2 * kPlaneStages + 2 + b); };
    auto bar_sums_full = [&](int b) { return bars + 8u * (2 * kPackedStages + 2 * kPlaneStages + 4 + b); };
    auto bar_sums_empty = [&](int b) { return bars + 8u * (2 * kPackedStages + 2 * kPlaneStages + 6 + b); };
    const uint32_t bar_drain = bars + 8u * (2 * kPackedStages + 2 * kPlaneStages + 8);
    const uint32_t bar_never = bars + 8u * (2 * kPackedStages + 2 * kPlaneStages + 9);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kSmMisc);
    volatile int *abort = reinterpret_cast<volatile int *>(smem + kSmMisc + 8);
    volatile int *epi_ok = reinterpret_cast<volatile int *>(smem + kSmMisc + 16);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kPackedStages; ++s) {
            mbar_init(bar_packed_full(s), 1);
            mbar_init(bar_packed_empty(s), kTeamWarps + (kBeam ? kBeamWarps : 0));
        }
        for (int s = 0; s < kPlaneStages; ++s) {
            mbar_init(bar_plane_full(s), kTeamWarps);
            mbar_init(bar_plane_empty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar_acc_full(b), 1);
            mbar_init(bar_acc_empty(b), kEpiWarps);
            mbar_init(bar_sums_full(b), kConvWarps);
            mbar_init(bar_sums_empty(b), kEpiWarps);
        }
        mbar_init(bar_drain, 1);
        mbar_init(bar_never, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int a = 0; a < p.n_arrays; ++a)
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmaps.m[a])) : "memory");
    }
    for (int e = threadIdx.x; e < kSumsBytes / 4; e += blockDim.x) sums[e] = 0;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const int first_item = blockIdx.x, item_step = gridDim.x;

    if (warp == 0) {
        // ------------------------------------------------- TMA producer --
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t issued = 0, issued_phase = 0;   // per slot: a load was issued / its parity
            bool ok = true;
            for (int item = first_item; ok && item < p.n_items; item += item_step) {
                const Item it = decode_item(p, item);
                const int n_stages = p.a[it.a].n_stages;
                const CUtensorMap *tmap = &tmaps.m[it.a];
                const int f = it.f, I = it.I, J = it.J;
                const bool diag = it.diag;
                // the item's first stages were prefetched during the previous
                // item (the first item's here); its later ones run ahead below,
                // and its last ones prefetch the next item's first
                if (item == first_item)
                    for (int s = 0; s < kPrefetchStages && s < n_stages; ++s) {
                        tma_prefetch_3d(tmap, I * kTile, f, s * kTc);
                        if (!diag) tma_prefetch_3d(tmap, J * kTile, f, s * kTc);
                    }
                const int nitem = item + item_step;
                Item nit{};
                int n_nst = 0;
                const CUtensorMap *ntmap = nullptr;
                if (nitem < p.n_items) {
                    nit = decode_item(p, nitem);
                    n_nst = p.a[nit.a].n_stages;
                    ntmap = &tmaps.m[nit.a];
                }
                for (int s = 0; s < n_stages; ++s) {
                    if (s + kPrefetchStages < n_stages) {
                        tma_prefetch_3d(tmap, I * kTile, f, (s + kPrefetchStages) * kTc);
                        if (!diag) tma_prefetch_3d(tmap, J * kTile, f, (s + kPrefetchStages) * kTc);
                    } else if (s + kPrefetchStages - n_stages < n_nst) {
                        const int ns = s + kPrefetchStages - n_stages;
                        tma_prefetch_3d(ntmap, nit.I * kTile, nit.f, ns * kTc);
                        if (!nit.diag) tma_prefetch_3d(ntmap, nit.J * kTile, nit.f, ns * kTc);
                    }
                    if (!mbar_wait(bar_packed_empty(stage), phase ^ 1u, abort, p.status, 1, p.wait_limit)) {
                        ok = false;
                        break;
                    }
                    const uint32_t full = bar_packed_full(stage);
                    const uint32_t dst = sbase + kSmPacked + stage * kPackedStageBytes;
                    mbar_expect_tx(full, diag ? kPackedTileBytes : 2 * kPackedTileBytes);
                    // upper half: the B tile (I); lower half: the A tile (J)
                    tma_load_3d(dst + kPackedTileBytes, tmap, full, I * kTile, f, s * kTc);
                    if (!diag) tma_load_3d(dst, tmap, full, J * kTile, f, s * kTc);
                    issued |= 1u << stage;
                    issued_phase = (issued_phase & ~(1u << stage)) | (phase << stage);
                    if (++stage == kPackedStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            // every issued load must have landed before the CTA may exit
            for (int k = 0; k < kPackedStages; ++k) {
                if (!((issued >> k) & 1u)) continue;
                const long long t0 = clock64();
                while (!mbar_try(bar_packed_full(k), (issued_phase >> k) & 1u) && clock64() - t0 < p.wait_limit) {
                }
            }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------- MMA issuer --
        if (lane == 0) {
            const uint64_t desc_planes = smem_desc(sbase + kSmPlanes, kPlaneBytes, 1024);
            int stage = 0;
            uint32_t phase = 0;
            // TMEM holds two accumulators ("slots"); a pair item fills both (its
            // diagonal part first), any other item the next one
            uint32_t slot_phase = 0;                 // bit s: phase of slot s
            int next_slot = 0;
            bool ok = true;
            for (int item = first_item; ok && item < p.n_items; item += item_step) {
                const Item it = decode_item(p, item);
                const int n_stages = p.a[it.a].n_stages;
                const bool pair = it.kind == kPairItem;
                const int s0 = next_slot, s1 = next_slot ^ 1;
                if (!pair) next_slot ^= 1;
                const int n_parts = pair ? 2 : 1;
                for (int part = 0; ok && part < n_parts; ++part) {
                    const int sl = part == 0 ? s0 : s1;
                    if (!mbar_wait(bar_acc_empty(sl), ((slot_phase >> sl) & 1u) ^ 1u, abort, p.status, 2,
                                   p.wait_limit))
                        ok = false;
                    slot_phase ^= 1u << sl;
                }
                if (!ok) break;
                fence_after();
                // descriptors differ only in the start-address field (bits 0-13,
                // address >> 4, below 2^14 for any shared address): build the
                // plane-stage-0 descriptors once and add offsets.  Part 0 of a pair
                // (and a diagonal item) multiplies the J planes by themselves.
                const bool a_is_b = it.kind != kOffItem;
                const uint32_t t0 = tmem + uint32_t(s0 * 256), t1 = tmem + uint32_t(s1 * 256);
                const uint64_t dR0 = desc_planes + uint64_t((a_is_b ? kOffRB : kOffRA) >> 4);
                const uint64_t dM0 = desc_planes + uint64_t((a_is_b ? kOffMB : kOffMA) >> 4);
                const uint64_t dR1 = desc_planes + uint64_t(kOffRA >> 4), dM1 = desc_planes + uint64_t(kOffMA >> 4);
                const uint64_t dRJ = desc_planes + uint64_t(kOffRB >> 4), dMJ = desc_planes + uint64_t(kOffMB >> 4);
                uint32_t accum = 0;
                if (pair) {
                    for (int s = 0; s < n_stages; ++s) {
                        if (!mbar_wait(bar_plane_full(stage), phase, abort, p.status, 3, p.wait_limit)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        const uint64_t so = uint64_t((stage * kPlaneStageBytes) >> 4);
                        mma_f8(t0, dR0 + so, dRJ + so, accum);
                        mma_f8(t0, dM0 + so, dMJ + so, 1);
                        mma_f8(t0, dR0 + so + 256u, dRJ + so + 256u, 1);
                        mma_f8(t0, dM0 + so + 256u, dMJ + so + 256u, 1);
                        mma_f8(t1, dR1 + so, dRJ + so, accum);
                        mma_f8(t1, dM1 + so, dMJ + so, 1);
                        mma_f8(t1, dR1 + so + 256u, dRJ + so + 256u, 1);
                        mma_f8(t1, dM1 + so + 256u, dMJ + so + 256u, 1);
                        accum = 1;
                        mma_commit(bar_plane_empty(stage));
                        if (++stage == kPlaneStages) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                } else {
                    for (int s = 0; s < n_stages; ++s) {
                        if (!mbar_wait(bar_plane_full(stage), phase, abort, p.status, 3, p.wait_limit)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        const uint64_t so = uint64_t((stage * kPlaneStageBytes) >> 4);
                        mma_f8(t0, dR0 + so, dRJ + so, accum);
                        mma_f8(t0, dM0 + so, dMJ + so, 1);
                        mma_f8(t0, dR0 + so + 256u, dRJ + so + 256u, 1);
                        mma_f8(t0, dM0 + so + 256u, dMJ + so + 256u, 1);
                        accum = 1;
                        mma_commit(bar_plane_empty(stage));
                        if (++stage == kPlaneStages) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                }
                if (!ok) break;
                mma_commit(bar_acc_full(s0));
                if (pair) mma_commit(bar_acc_full(s1));
            }
            // drain all MMAs issued by this thread before TMEM is released
            mma_commit(bar_drain);
            const long long t0 = clock64();
            while (!mbar_try(bar_drain, 0) && clock64() - t0 < p.wait_limit) {
            }
        }
    } else if ((warp >= 2 && warp <= 16) || warp == 22) {
        // ----------------------------------------------------- converters --
        // Two teams of kTeamWarps warps; team t converts the stages g (counted
        // over all items of this CTA) with g % 2 == t, so each warp spends its
        // barrier latency once per two stages.  Thread u of a team owns chunk
        // column c (16 inputs) of one tile and a set of rows of each of its
        // stages, so its per-input sums cover 16 inputs and stay in registers:
        //   off-diagonal item: q < 16 -> B tile, q >= 16 -> A tile, rows (q & 15) + 16k, k < 4
        //   diagonal item:     B tile, rows q + 32k, k < 2
        // The B tile (upper half of the packed stage) becomes the planes M, R and
        // -M, the A tile (lower half) R and M; a diagonal item's single tile is
        // both, as B.
        const int ci = warp <= 16 ? warp - kFirstConvWarp : 15;
        const int team = ci / kTeamWarps;
        const int u = (ci % kTeamWarps) * 32 + lane;   // 0..255
        const int c = u & 7, q = u >> 3;                                         // q 0..31
        uint32_t g0 = 0;                        // global index of the item's first stage
        int local = 0;
        bool ok = true;
        for (int item = first_item; ok && item < p.n_items; item += item_step, ++local) {
            const Item it = decode_item(p, item);
            const int n_stages = p.a[it.a].n_stages;
            const bool diag = it.diag;
            const bool tile_b = diag || q < 16;
            const int n_units = diag ? 2 : 4;
            const int row0 = diag ? q : (q & 15), row_step = diag ? 32 : 16;
            const uint32_t src_tile = tile_b ? uint32_t(kPackedTileBytes) : 0u;
            // per-input code sums of this thread's 16 inputs: byte lanes
            // (<= 16 rows of codes <= 15 between widenings), then 16-bit lanes
            uint32_t b8[2][4], s16lo[2][4], s16hi[2][4];
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int k = 0; k < 4; ++k) b8[m][k] = s16lo[m][k] = s16hi[m][k] = 0;
            int since_widen = 0;
            const uint32_t first = g0 + uint32_t((team - int(g0 & 1u)) & 1);
            for (uint32_t gg = first; gg < g0 + uint32_t(n_stages); gg += 2) {
                const int pstage = int(gg % kPackedStages), cstage = int(gg % kPlaneStages);
                const uint32_t pphase = (gg / kPackedStages) & 1u, cphase = (gg / kPlaneStages) & 1u;
                if (!mbar_wait(bar_packed_full(pstage), pphase, abort, p.status, 4, p.wait_limit) ||
                    !mbar_wait(bar_plane_empty(cstage), cphase ^ 1u, abort, p.status, 5, p.wait_limit)) {
                    ok = false;
                    break;
                }
                const uint8_t *pk = smem + kSmPacked + pstage * kPackedStageBytes + src_tile;
                uint8_t *pl = smem + kSmPlanes + cstage * kPlaneStageBytes;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (k >= n_units) break;
                    const int row = row0 + k * row_step;
                    const uint4 w = *reinterpret_cast<const uint4 *>(pk + row * 128 + c * 16);
                    const uint32_t so = uint32_t(row * 128 + ((c ^ (row & 7)) << 4));
                    const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
                    uint32_t R[4], M[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        codes(ww[e], kZeroInvalid, R[e], M[e]);
                        b8[0][e] += R[e];
                        b8[1][e] += M[e];
                    }
                    if (tile_b) {
                        *reinterpret_cast<uint4 *>(pl + kOffMB + so) = make_uint4(M[0], M[1], M[2], M[3]);
                        *reinterpret_cast<uint4 *>(pl + kOffRB + so) = make_uint4(R[0], R[1], R[2], R[3]);
                        *reinterpret_cast<uint4 *>(pl + kOffNMB + so) =
                            make_uint4(M[0] | 0x80808080u, M[1] | 0x80808080u, M[2] | 0x80808080u,
                                       M[3] | 0x80808080u);
                    } else {
                        *reinterpret_cast<uint4 *>(pl + kOffRA + so) = make_uint4(R[0], R[1], R[2], R[3]);
                        *reinterpret_cast<uint4 *>(pl + kOffMA + so) = make_uint4(M[0], M[1], M[2], M[3]);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(bar_plane_full(cstage));
                    mbar_arrive(bar_packed_empty(pstage));
                }

                // byte lanes: at most 4 stages x 4 rows of codes <= 15 (240)
                if (++since_widen == 4) {
                    since_widen = 0;
#pragma unroll
                    for (int m = 0; m < 2; ++m)
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            s16lo[m][k] += b8[m][k] & 0x00FF00FFu;
                            s16hi[m][k] += (b8[m][k] >> 8) & 0x00FF00FFu;
                            b8[m][k] = 0;
                        }
                }
            }
            if (!ok) break;
            g0 += uint32_t(n_stages);
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    s16lo[m][k] += b8[m][k] & 0x00FF00FFu;
                    s16hi[m][k] += (b8[m][k] >> 8) & 0x00FF00FFu;
                }
            // reduce over the four lanes of this warp that share chunk column c
            // and tile (16-bit lanes stay below 4 x 256 x 4 x 15 < 2^16), then
            // hand the per-input sums of this item to the epilogue
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    s16lo[m][k] += __shfl_xor_sync(0xFFFFFFFFu, s16lo[m][k], 8);
                    s16lo[m][k] += __shfl_xor_sync(0xFFFFFFFFu, s16lo[m][k], 16);
                    s16hi[m][k] += __shfl_xor_sync(0xFFFFFFFFu, s16hi[m][k], 8);
                    s16hi[m][k] += __shfl_xor_sync(0xFFFFFFFFu, s16hi[m][k], 16);
                }
            const int buf = local & 1;
            if (!warp_wait(bar_sums_empty(buf), ((local >> 1) & 1) ^ 1, abort, p.status, 6, lane, p.wait_limit, 64)) {
                ok = false;
                break;
            }
            if (lane < 8) {
                int *sb = sums + buf * (2 * 2 * kTile) + (tile_b ? 1 : 0) * 2 * kTile;
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    int *row_sums = sb + m * kTile;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int n0 = c * 16 + 4 * k;
                        atomicAdd(row_sums + sum_slot(n0 + 0), int(s16lo[m][k] & 0xFFFFu));
                        atomicAdd(row_sums + sum_slot(n0 + 1), int(s16hi[m][k] & 0xFFFFu));
                        atomicAdd(row_sums + sum_slot(n0 + 2), int(s16lo[m][k] >> 16));
                        atomicAdd(row_sums + sum_slot(n0 + 3), int(s16hi[m][k] >> 16));
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_sums_full(buf));
        }
    } else if (kBeam && warp >= kFirstBeamWarp) {
        // --------------------------------------------------- incoherent beam --
        // Every tile's 128 inputs are added once per channel and sample: the
        // B tile of each diagonal item (single items) or pair item, and for the
        // pair item (1, 0) its A tile (0) too, which the diagonal item (0, 0)
        // then leaves out.  Beam warp w takes tile B (w < 2) or A (w >= 2);
        // its lane l owns row 32 (w mod 2) + l of each stage (a sample) and
        // reads its 8 chunks rotated by l, so the 8 lanes of a quarter-warp
        // always hit 8 different 16-byte bank groups.  The warps walk every
        // stage of the CTA in order and release each packed slot with the
        // converters.
        const int bw = warp - kFirstBeamWarp;
        const int row = (bw & 1) * 32 + lane;
        const bool upper = bw < 2;                      // the B tile, in the upper half of the packed stage
        uint32_t g0 = 0;
        bool ok = true;
        for (int item = first_item; ok && item < p.n_items; item += item_step) {
            const Item it = decode_item(p, item);
            const ArrayParams &A = p.a[it.a];
            const int n_stages = A.n_stages;
            const bool pairs = A.pairs != 0 && A.n_tiles > 1;
            const bool b_tile = A.beam && (it.kind == kPairItem || (it.kind == kDiagItem && !pairs));
            const bool a_tile = A.beam && it.kind == kPairItem && it.J == 0;
            int32_t *const beam_f = A.beam ? A.beam + it.f : nullptr;
            for (uint32_t gg = g0; gg < g0 + uint32_t(n_stages); ++gg) {
                const int pstage = int(gg % kPackedStages);
                const uint32_t pphase = (gg / kPackedStages) & 1u;
                int okw = 1;
                if (lane == 0) okw = mbar_wait(bar_packed_full(pstage), pphase, abort, p.status, 10, p.wait_limit);
                okw = __shfl_sync(0xFFFFFFFFu, okw, 0);
                if (!okw) {
                    ok = false;
                    break;
                }
                (void)mbar_try(bar_packed_full(pstage), pphase);   // completed: acquire for every lane
                const int t = int(gg - g0) * kTc + row;
                if ((upper ? b_tile : a_tile) && t < A.nt) {
                    const uint8_t *src = smem + kSmPacked + pstage * kPackedStageBytes + row * 128 +
                                         (upper ? kPackedTileBytes : 0);
                    // four independent sums (one per word of a chunk) keep the
                    // dp4a chains short
                    int a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const uint4 w = *reinterpret_cast<const uint4 *>(src + ((k + lane) & 7) * 16);
                        a0 = power256(w.x, kZeroInvalid, a0);
                        a1 = power256(w.y, kZeroInvalid, a1);
                        a2 = power256(w.z, kZeroInvalid, a2);
                        a3 = power256(w.w, kZeroInvalid, a3);
                    }
                    atomicAdd(beam_f + (size_t)((A.beam_t0 + t) / A.beam_avg) * A.beam_ld, (a0 + a1 + a2 + a3) >> 8);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_packed_empty(pstage));
            }
            g0 += uint32_t(n_stages);
        }
    } else if (warp >= kFirstEpiWarp && warp < kFirstEpiWarp + kEpiWarps) {
        // ------------------------------------------------------- epilogue --
        const int q = warp & 3;                      // TMEM lane quarter of this warp
        uint32_t slot_phase = 0;                      // bit s: phase of TMEM slot s (same rule as the MMA warp)
        int next_slot = 0;
        int local = 0;
        bool ok = true;
        if (p.inject_stall) {
            // test hook: a wait that nothing ever satisfies; it must expire, record
            // CORR_E_TIMEOUT and take every role of the CTA down the abort path
            const bool mine = warp_wait(bar_never, 0, abort, p.status, 9, lane, p.wait_limit, 64);
            if (lane == 0) epi_ok[q] = mine ? 1 : 0;
            named_sync(2, kEpiWarps * 32);
            ok = epi_ok[0] && epi_ok[1] && epi_ok[2] && epi_ok[3];
            named_sync(2, kEpiWarps * 32);
        }
        for (int item = first_item; ok && item < p.n_items; item += item_step, ++local) {
            const Item it = decode_item(p, item);
            // copy this array's parameters into registers once per item
            const int n_in = p.a[it.a].n;
            const bool fresh = p.a[it.a].fresh != 0;
            int32_t *const acc = p.a[it.a].acc;
            const long long P = n_pairs(n_in);
            const int T_eff = p.a[it.a].n_stages * kTc;
            const int f = it.f;
            const bool pair = it.kind == kPairItem;
            const int s0 = next_slot, s1 = next_slot ^ 1;
            if (!pair) next_slot ^= 1;
            const int sbuf = local & 1;
            int *sb = sums + sbuf * (2 * 2 * kTile);               // A tile sums: [r/m][slot]
            int *sbB = sb + 1 * 2 * kTile;                         // B tile sums
            // TMEM lane a of a part holds input a of its A tile (an output column
            // j), TMEM column b (Re) and 128 + b (Im) input b of the B tile (an
            // output row i): D[a][b] = sum x_a conj(x_b), so V_ij = conj(D[a][b]).
            // This thread's input a in either tile gives its row terms (E, D of the
            // offset corrections), read before the B sums become column terms.
            int EaA = 0, DaA = 0, EaB = 0, DaB = 0;
            const int il = q * 32 + lane;
            const size_t out_f = (size_t)f * P;
            const int n_parts = pair ? 2 : 1;
            for (int part = 0; part < n_parts; ++part) {
                const int sl = part == 0 ? s0 : s1;
                // part 0 of a pair, or a diagonal item: the B tile against itself
                const bool dpart = part == 0 ? it.kind != kOffItem : false;
                const int At = dpart ? it.I : it.J;
                // the four epilogue warps decide together whether to go on, so that
                // none of them is ever left waiting at a named barrier
                bool mine = warp_wait(bar_acc_full(sl), (slot_phase >> sl) & 1u, abort, p.status, 7, lane,
                                      p.wait_limit, 256);
                if (part == 0)
                    mine = mine && warp_wait(bar_sums_full(sbuf), uint32_t(local >> 1) & 1u, abort, p.status, 8,
                                             lane, p.wait_limit, 64);
                if (lane == 0) epi_ok[q] = mine ? 1 : 0;
                named_sync(2, kEpiWarps * 32);
                ok = epi_ok[0] && epi_ok[1] && epi_ok[2] && epi_ok[3];
                if (ok && part == 0) {
                    const int SrB = sbB[sum_slot(il)], SmB = sbB[kTile + sum_slot(il)];
                    const int SrA = sb[sum_slot(il)], SmA = sb[kTile + sum_slot(il)];
                    EaB = SrB + SmB;
                    DaB = SmB - SrB;
                    EaA = SrA + SmA;
                    DaA = SmA - SrA;
                    named_sync(2, kEpiWarps * 32);
                    // input b's column terms, as floats in column order (the B sums
                    // area holds exactly 2 x 128 floats): -8 E_b for Re in the first
                    // half, -8 D_b for Im in the second, so that two adjacent columns'
                    // terms are one float pair for the paired arithmetic below
                    reinterpret_cast<float *>(sbB)[il] = float(-8 * EaB);
                    reinterpret_cast<float *>(sbB)[kTile + il] = float(-8 * DaB);
                }
                named_sync(2, kEpiWarps * 32);
                if (!ok) break;
                slot_phase ^= 1u << sl;
                fence_after();
                const int j = At * kTile + il;                     // this lane's output column
                const int Ea = dpart ? EaB : EaA, Da = dpart ? DaB : DaA;
                // Re V_ij = P_re - 8 E_b + (128 T - 8 E_a) and Im V_ij = -P'_im - 8 D_b + 8 D_a,
                // with P' the TMEM product (Im of x_a conj(x_b)) and b = i, a = j:
                // computed in fp32 on integer values (TMEM * 2^18 is the integer
                // product sum, every partial sum is below 2^24 in magnitude, so each
                // step is exact), and adding 1.5 * 2^23 leaves V (|V| <= 128 T <=
                // 2^22) as the low bits of the float's encoding
                const float row_re = float(128 * T_eff - 8 * Ea) + 12582912.0f;
                const float row_im = float(8 * Da) + 12582912.0f;
                const float4 *colre = reinterpret_cast<const float4 *>(sbB);          // -8 E_b, b = 4 m .. 4 m + 3
                const float4 *colim = reinterpret_cast<const float4 *>(sbB + kTile);  // -8 D_b
                const uint32_t taddr = tmem + uint32_t(sl * 256) + (uint32_t(q * 32) << 16);
                const int i0 = it.I * kTile;
                // in the diagonal part, column b holds output row i0 + b, whose
                // columns j <= i: chunks wholly left of this warp's lanes are skipped;
                // in a launch that stores, warp 0 leaves its blocks of rows 64-127 to
                // warps 2 and 3 (below), so that no warp drains more than 12 of the
                // part's 40 chunk-columns (a launch that adds keeps every add coalesced;
                // the beam variant, bound by its beam warps, keeps its registers)
                const bool split = !kBeam && dpart && fresh;
                const int c_first = dpart ? ((32 * q) & ~7) : 0;
                const int c_last = split && q == 0 ? 64 : kTile;
                int2 *const colp = reinterpret_cast<int2 *>(acc) + out_f + j;
#pragma unroll 1
                for (int c0 = c_first; c0 < c_last && i0 + c0 < n_in; c0 += 8) {
                    uint32_t vre[8], vim[8];
                    tmem_ld8(taddr + c0, vre);
                    tmem_ld8(taddr + 128 + c0, vim);
                    // element k: output row i = ic + k, column j (this lane):
                    // consecutive lanes write consecutive elements of the row
                    const int ic = i0 + c0;
                    int2 *const p0 = colp + (size_t)(unsigned(ic) * unsigned(ic + 1) / 2u);
                    const bool full = ic + 7 < n_in && (!dpart || c0 >= 32 * q + 32);
                    int2 v[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) v[k] = make_int2(0, 0);
                    tmem_wait_ld();
#pragma unroll
                    for (int k = 0; k < 8; k += 4) {
                        // paired fp32 (sm_100+): each instruction does two columns
                        const float4 cr = colre[(c0 + k) >> 2], ci = colim[(c0 + k) >> 2];
#pragma unroll
                        for (int e = 0; e < 4; e += 2) {
                            const float2 re = __fadd2_rn(
                                __ffma2_rn(make_float2(__uint_as_float(vre[k + e]), __uint_as_float(vre[k + e + 1])),
                                           make_float2(262144.0f, 262144.0f),
                                           e == 0 ? make_float2(cr.x, cr.y) : make_float2(cr.z, cr.w)),
                                make_float2(row_re, row_re));
                            const float2 im = __fadd2_rn(
                                __ffma2_rn(make_float2(__uint_as_float(vim[k + e]), __uint_as_float(vim[k + e + 1])),
                                           make_float2(-262144.0f, -262144.0f),
                                           e == 0 ? make_float2(ci.x, ci.y) : make_float2(ci.z, ci.w)),
                                make_float2(row_im, row_im));
                            v[k + e].x += __float_as_int(re.x) - 0x4B400000;
                            v[k + e + 1].x += __float_as_int(re.y) - 0x4B400000;
                            v[k + e].y += __float_as_int(im.x) - 0x4B400000;
                            v[k + e + 1].y += __float_as_int(im.y) - 0x4B400000;
                        }
                    }
                    int2 *pk = p0;
                    if (!fresh) {
                        // a launch that adds into the output: the integer adds are done
                        // in L2 (red), so no warp waits on reading the eight scattered
                        // row pieces of a chunk back first
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            if (full || (ic + k < n_in && (!dpart || il <= c0 + k))) {
                                asm volatile("red.global.add.s32 [%0], %1;" ::"l"(&pk->x), "r"(v[k].x) : "memory");
                                asm volatile("red.global.add.s32 [%0], %1;" ::"l"(&pk->y), "r"(v[k].y) : "memory");
                            }
                            pk += ic + k + 1;
                        }
                    } else if (full) {
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            *pk = v[k];
                            pk += ic + k + 1;
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            if (ic + k < n_in && (!dpart || il <= c0 + k)) *pk = v[k];
                            pk += ic + k + 1;
                        }
                    }
                }
                if (split && q >= 2 && i0 + 32 * q < n_in) {
                    // rows 32 q .. 32 q + 31, columns 0-31 of the diagonal block from this
                    // warp's own lanes: here TMEM lane a is output row i and column b output
                    // column j < 32 <= i, and D[a][b] = V_ij itself (Im with the other sign
                    // of the D terms); each lane writes 8 consecutive elements of its row.
                    // The TMEM loads are warp-wide: the condition above is the warp's,
                    // the one below each lane's
                    const int i = i0 + il;
                    const bool live = i < n_in;
                    const float rrow_im = float(-8 * Da) + 12582912.0f;
                    int2 *const rowp = reinterpret_cast<int2 *>(acc) + out_f + (size_t)i * (i + 1) / 2 + i0;
#pragma unroll 1
                    for (int c0 = 0; c0 < 32; c0 += 8) {
                        uint32_t vre[8], vim[8];
                        tmem_ld8(taddr + c0, vre);
                        tmem_ld8(taddr + 128 + c0, vim);
                        tmem_wait_ld();
                        int2 v[8];
#pragma unroll
                        for (int k = 0; k < 8; k += 4) {
                            const float4 cr = colre[(c0 + k) >> 2], ci = colim[(c0 + k) >> 2];
#pragma unroll
                            for (int e = 0; e < 4; e += 2) {
                                const float2 re = __fadd2_rn(
                                    __ffma2_rn(make_float2(__uint_as_float(vre[k + e]), __uint_as_float(vre[k + e + 1])),
                                               make_float2(262144.0f, 262144.0f),
                                               e == 0 ? make_float2(cr.x, cr.y) : make_float2(cr.z, cr.w)),
                                    make_float2(row_re, row_re));
                                const float2 im = __fadd2_rn(
                                    __ffma2_rn(make_float2(__uint_as_float(vim[k + e]), __uint_as_float(vim[k + e + 1])),
                                               make_float2(262144.0f, 262144.0f),
                                               e == 0 ? make_float2(-ci.x, -ci.y) : make_float2(-ci.z, -ci.w)),
                                    make_float2(rrow_im, rrow_im));
                                v[k + e].x = __float_as_int(re.x) - 0x4B400000;
                                v[k + e + 1].x = __float_as_int(re.y) - 0x4B400000;
                                v[k + e].y = __float_as_int(im.x) - 0x4B400000;
                                v[k + e + 1].y = __float_as_int(im.y) - 0x4B400000;
                            }
                        }
                        int2 *const dst = rowp + c0;
                        if (!live) {
                        } else if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
                            for (int k = 0; k < 8; k += 2)
                                *reinterpret_cast<int4 *>(dst + k) = make_int4(v[k].x, v[k].y, v[k + 1].x, v[k + 1].y);
                        } else {
                            dst[0] = v[0];
#pragma unroll
                            for (int k = 1; k < 7; k += 2)
                                *reinterpret_cast<int4 *>(dst + k) = make_int4(v[k].x, v[k].y, v[k + 1].x, v[k + 1].y);
                            dst[7] = v[7];
                        }
                    }
                }
                // this part's TMEM slot can take the next accumulation
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_acc_empty(sl));
            }
            if (!ok) break;
            // every epilogue warp has read this item's sums: clear them for the
            // item that reuses the buffer, then release it
            named_sync(2, kEpiWarps * 32);
            for (int e = threadIdx.x - kFirstEpiWarp * 32; e < 2 * 2 * kTile; e += kEpiWarps * 32) sb[e] = 0;
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_sums_empty(sbuf));
        }
    }

    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// ------------------------------------------------------------- host side --
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        else
            cudaGetLastError();
    });
    return g_encode;
}

int g_sm_count[64] = {0};
int g_attr_set[64] = {0};
std::mutex g_dev_mu;

}  // namespace

bool tc_supported(int n_inputs, int device)
{
    if (n_inputs < 1 || device < 0 || device >= 64) return false;
    static int cached[64] = {0};                 // 0 unknown, 1 yes, -1 no
    if (cached[device] == 0) {
        cudaDeviceProp prop;
        bool ok = cudaGetDeviceProperties(&prop, device) == cudaSuccess && prop.major == 10 &&
                  prop.minor == 3 && prop.sharedMemPerBlockOptin >= size_t(kSmemBytes) &&
                  encoder() != nullptr;
        cudaGetLastError();
        cached[device] = ok ? 1 : -1;
    }
    return cached[device] == 1;
}

cudaError_t launch_group(const TcArray *arrays, int count, bool zero_invalid, int dev,
                         DeviceStatus *status, const TcOptions &opt, cudaStream_t s);

cudaError_t launch_xeng_tc_batch(const TcArray *arrays, int count, DeviceStatus *status,
                                 const TcOptions &opt, cudaStream_t s)
{
    if (count < 0 || count > kMaxArrays) return cudaErrorInvalidValue;
    auto enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(g_dev_mu);
        if (!g_attr_set[dev]) {
            for (auto fn : {xeng_tc_kernel<false, false>, xeng_tc_kernel<true, false>, xeng_tc_kernel<false, true>,
                            xeng_tc_kernel<true, true>}) {
                e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
                if (e != cudaSuccess) return e;
            }
            e = cudaDeviceGetAttribute(&g_sm_count[dev], cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
            g_attr_set[dev] = 1;
        }
    }
    // arrays with work, longest items first; the invalid-sample mode is a
    // property of the kernel, so arrays with different modes go to different
    // launches
    for (int k = 0; k < count; ++k) {
        const TcArray &A = arrays[k];
        if (A.nt <= 0) continue;
        const int ld = A.ld ? A.ld : A.n;
        if (A.nt > kTcMaxSamples || A.n < 1 || ld < A.n || ld % 16 != 0 || A.n_chan < 1 || !A.acc ||
            (reinterpret_cast<uintptr_t>(A.volt) & 15) != 0)
            return cudaErrorInvalidValue;
    }
    for (int mode = 0; mode < 2; ++mode) {
        e = launch_group(arrays, count, mode == 1, dev, status, opt, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Channels [c0, c0 + chans) of one array, as one array of the launch.
struct Span {
    const TcArray *A;
    int c0, chans;
    bool pairs;
};

// Largest cost over the CTAs of the static schedule (CTA c takes items c, c +
// grid, ...), in half tile pairs of MMA work, with conversion counted in: a pair
// item (two tile pairs, two tiles converted) 4, an off-diagonal item (one tile
// pair, two tiles converted) 3, a diagonal item (one tile pair, one tile) 2.
long long schedule_max_cost(const Span *sp, int m, int grid)
{
    static thread_local long long cost[1024];
    const int g = grid < 1024 ? grid : 1024;
    for (int c = 0; c < g; ++c) cost[c] = 0;
    long long item = 0;
    for (int k = 0; k < m; ++k) {
        const int n_tiles = (sp[k].A->n + kTile - 1) / kTile;
        const bool pairs = sp[k].pairs;
        const int per_chan = items_per_channel(n_tiles, pairs);
        const bool rot = grid % per_chan == 0;
        const long long begin = item;
        for (long long local = 0; local < (long long)sp[k].chans * per_chan; ++local, ++item) {
            const long long f = local / per_chan;
            const int kk = int(local - f * per_chan);
            const long long round = (begin + f * per_chan) / grid;
            int I, J, kind;
            item_tiles(rot ? int((kk + round) % per_chan) : kk, n_tiles, pairs, I, J, kind);
            cost[item % g] += kind == kPairItem ? 4 : kind == kOffItem ? 3 : 2;
        }
    }
    long long mx = 0;
    for (int c = 0; c < g; ++c) mx = cost[c] > mx ? cost[c] : mx;
    return mx;
}

cudaError_t launch_group(const TcArray *arrays, int count, bool zero_invalid, int dev,
                         DeviceStatus *status, const TcOptions &opt, cudaStream_t s)
{
    auto enc = encoder();
    int order[kMaxArrays], m = 0;
    for (int k = 0; k < count; ++k)
        if (arrays[k].nt > 0 && arrays[k].zero_invalid == zero_invalid) order[m++] = k;
    if (m == 0) return cudaSuccess;
    for (int x = 1; x < m; ++x)
        for (int y = x; y > 0 && arrays[order[y]].nt > arrays[order[y - 1]].nt; --y) {
            const int t = order[y];
            order[y] = order[y - 1];
            order[y - 1] = t;
        }
    Span sp[kMaxArrays];
    long long items = 0;
    for (int k = 0; k < m; ++k) {
        const TcArray &A = arrays[order[k]];
        const int n_tiles = (A.n + kTile - 1) / kTile;
        const int n_stages = (A.nt + kTc - 1) / kTc;
        const bool want_pairs = A.items == TcItems::kPairs ||
                                (A.items == TcItems::kAuto && n_stages >= kPairMinStages);
        sp[k] = Span{&A, 0, A.n_chan, n_tiles > 1 && want_pairs};
        items += (long long)A.n_chan * items_per_channel(n_tiles, sp[k].pairs);
    }
    // The last round of the static schedule: where the last array runs pair
    // items, its last x channels may run as single items instead, x the fewest
    // channels that fill the last (partial) round with single items, so that a
    // CTA's extra item is one tile pair, not two; taken when it lowers the
    // largest cost of a CTA (for 256 inputs x 3072 channels on 152 SMs, x = 32:
    // 96 single items instead of 32 pair and 32 diagonal items).  Either
    // schedule computes the same sums: only the time differs.
    const int sms = g_sm_count[dev];
    if (sp[m - 1].pairs && m < kMaxArrays && items > sms && items <= (1 << 22)) {
        const Span last = sp[m - 1];
        const int n_tiles = (last.A->n + kTile - 1) / kTile;
        const int pp = items_per_channel(n_tiles, true), ps = items_per_channel(n_tiles, false);
        int x = 1;
        for (; x < last.chans; ++x) {
            const long long n2 = items + (long long)x * (ps - pp);
            const long long r = n2 % sms;
            if ((r ? r : sms) <= (long long)x * ps) break;
        }
        if (x < last.chans) {
            // the decision depends on the launch's shapes only: keep the last one
            struct Key {
                long long items;
                int sms, m, n, chans;
                bool take;
            };
            static thread_local Key memo{-1, 0, 0, 0, 0, false};
            const bool hit = memo.items == items && memo.sms == sms && memo.m == m && memo.n == last.A->n &&
                             memo.chans == last.chans;
            bool take = memo.take;
            sp[m - 1].chans = last.chans - x;
            sp[m] = Span{last.A, last.chans - x, x, false};
            if (!hit) {
                sp[m - 1] = last;
                const long long before = schedule_max_cost(sp, m, sms);
                sp[m - 1].chans = last.chans - x;
                take = schedule_max_cost(sp, m + 1, sms) < before;
                memo = Key{items, sms, m, last.A->n, last.chans, take};
            }
            if (take) {
                ++m;
                items += (long long)x * (ps - pp);
            } else {
                sp[m - 1] = last;
            }
        }
    }
    Tmaps maps;
    Params prm{};
    items = 0;
    for (int k = 0; k < m; ++k) {
        const TcArray &A = *sp[k].A;
        const int c0 = sp[k].c0;
        // extent n along the inputs: a box reaching past it (a ragged last tile)
        // reads zero bytes, i.e. samples 0 + 0i, which cancel in the corrections
        const cuuint64_t ld = cuuint64_t(A.ld ? A.ld : A.n);
        const cuuint64_t dims[3] = {cuuint64_t(A.n), cuuint64_t(sp[k].chans), cuuint64_t(A.nt)};
        const cuuint64_t strides[2] = {ld, ld * cuuint64_t(A.n_chan)};
        const cuuint32_t box[3] = {cuuint32_t(kTile), 1u, cuuint32_t(kTc)};
        const cuuint32_t estr[3] = {1u, 1u, 1u};
        CUresult cr = enc(&maps.m[k], CU_TENSOR_MAP_DATA_TYPE_UINT8, 3,
                          const_cast<uint8_t *>(A.volt) + size_t(c0) * ld, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
        ArrayParams &P = prm.a[k];
        P.acc = A.acc + size_t(c0) * size_t(n_pairs(A.n)) * 2;
        P.n = A.n;
        P.n_chan = sp[k].chans;
        P.nt = A.nt;
        P.n_tiles = (A.n + kTile - 1) / kTile;
        P.n_stages = (A.nt + kTc - 1) / kTc;
        P.item_begin = int(items);
        P.fresh = A.fresh ? 1 : 0;
        P.pairs = sp[k].pairs ? 1 : 0;
        P.per_chan = items_per_channel(P.n_tiles, P.pairs != 0);
        P.beam = A.beam ? A.beam + c0 : nullptr;
        P.beam_ld = A.n_chan;
        P.beam_avg = A.beam_avg > 0 ? A.beam_avg : 1;
        P.beam_t0 = A.beam_t0;
        items += (long long)sp[k].chans * P.per_chan;
    }
    if (items > 0x7FFFFFFF) return cudaErrorInvalidValue;
    prm.n_arrays = m;
    prm.n_items = int(items);
    prm.status = status;
    prm.wait_limit = opt.wait_limit > 0 ? opt.wait_limit : kDefaultWaitLimit;
    prm.inject_stall = opt.inject_stall ? 1 : 0;
    const int grid = prm.n_items < g_sm_count[dev] ? prm.n_items : g_sm_count[dev];
    for (int k = 0; k < m; ++k) {
        ArrayParams &P = prm.a[k];
        P.rot_step = grid % P.per_chan == 0 ? 1 : 0;
    }
    bool beam = false;
    for (int k = 0; k < m; ++k) beam = beam || prm.a[k].beam != nullptr;
    const int threads = beam ? kThreadsBeam : kThreads;
    if (zero_invalid)
        (beam ? xeng_tc_kernel<true, true> : xeng_tc_kernel<true, false>)<<<grid, threads, kSmemBytes, s>>>(maps,
                                                                                                           prm);
    else
        (beam ? xeng_tc_kernel<false, true> : xeng_tc_kernel<false, false>)<<<grid, threads, kSmemBytes, s>>>(
            maps, prm);
    return cudaGetLastError();
}

}  // namespace corr
