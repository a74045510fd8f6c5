// C ABI of the X-engine library: context, workspace, integration control,
// host-buffer transfers, checkpoint/resume and errors (declared in corr.h).
//
// Call structure of one integration (Section 3.4.1: a block of input is
// released to the GPU; Section 3.4.3: products accumulate on the device and
// are copied out at the end of the operator-chosen accumulation length):
//
//   corr_accumulate(volt)  -> [unpack K1 ->] X-engine K2 into the int32
//                             packed-triangle accumulators (all on `stream`)
//   corr_dump(vis)         -> K3 copy, accumulators marked fresh
//
// Nothing here synchronises the host except corr_sync and the state calls.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.cuh"

using namespace corr;

namespace {
// NVTX range around a public call (free when no profiler is attached): the
// unpack, X-engine and dump launches show up under the call that made them.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};
}  // namespace

struct corr_ctx {
    int n = 0, f = 0, t_max = 0;
    int device = 0, sm_major = 0, sm_minor = 0, sm_count = 0;
    int path = CORR_PATH_AUTO;
    int tile = 0;            // CUDA-core tile (32 or 64) or tcgen05 items (128, 256); 0 = chosen by shape
    long long wait_limit = 0;   // device bounded-wait limit (cycles), 0 = default
    bool inject_stall = false;  // one-shot test hook for the next tensor-core launch
    unsigned flags = 0;

    // workspace (caller-owned device memory)
    uint8_t *ws = nullptr;
    size_t ws_bytes = 0;
    DeviceStatus *status = nullptr;
    int32_t *acc = nullptr;
    uint8_t *stage = nullptr;
    uint8_t *host_stage[kHostBuffers] = {};
    uint8_t *tc_pad = nullptr;   // 16-byte-aligned rows for the tensor-core path (n % 16 != 0)

    StagePlan dp4a{}, mma{};
    int host_chunk = 0;
    int host_next = 0;     // staging buffer of the next host chunk (rotates across calls)

    long long samples = 0;
    bool fresh = true;     // accumulators hold no data: next X-engine stores

    cudaStream_t copy_stream = nullptr;             // host -> device chunk copies
    cudaEvent_t ev_full[kHostBuffers] = {};
    cudaEvent_t ev_free[kHostBuffers] = {};
    cudaStream_t out_stream = nullptr;              // device -> host dump copies
    cudaEvent_t ev_dumped = nullptr, ev_out_free = nullptr;
    bool out_pending = false;  // a host dump may still be reading the accumulators

    // profiling: launch counts (always) and event pairs (when enabled)
    bool prof_on = false;
    long long prof_launches[CORR_K_KINDS] = {0, 0, 0, 0};
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pending[CORR_K_KINDS];
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pool;
    std::pair<cudaEvent_t, cudaEvent_t> prof_cur{nullptr, nullptr};
};

namespace {

thread_local int g_last_error = CORR_OK;

int ret(int status)
{
    g_last_error = status;
    return status;
}

struct WsLayout {
    size_t status_off, acc_off, stage_off, host_off[kHostBuffers], pad_off, total;
};

// Row stride of the tensor-core path's padded copy, and the samples one copy
// holds (0 when the rows need no padding).
int tc_ld(int n) { return int(round_up(size_t(n), 16)); }
int tc_pad_samples(int n, int n_chan, int t_max)
{
    if (n % 16 == 0) return 0;
    const size_t row = size_t(tc_ld(n)) * size_t(n_chan);
    size_t t = kTcPadCap / row / 64 * 64;
    if (t < 64) t = 64;
    const size_t whole = round_up(size_t(t_max), 64);
    return int(t < whole ? t : whole);
}

size_t acc_words(const corr_ctx *c) { return size_t(c->f) * size_t(n_pairs(c->n)) * 2; }

WsLayout layout_of(const corr_ctx *c)
{
    WsLayout L{};
    size_t off = 0;
    L.status_off = off;
    off = round_up(off + sizeof(DeviceStatus), kAlign);
    L.acc_off = off;
    off = round_up(off + acc_words(c) * sizeof(int32_t), kAlign);
    L.stage_off = off;
    const size_t stage = c->dp4a.bytes > c->mma.bytes ? c->dp4a.bytes : c->mma.bytes;
    off = round_up(off + stage, kAlign);
    const size_t host = size_t(c->host_chunk) * size_t(c->f) * size_t(c->n);
    for (int b = 0; b < kHostBuffers; ++b) {
        L.host_off[b] = off;
        off = round_up(off + host, kAlign);
    }
    L.pad_off = off;
    off = round_up(off + size_t(tc_pad_samples(c->n, c->f, c->t_max)) * size_t(tc_ld(c->n)) * size_t(c->f),
                   kAlign);
    L.total = off;
    return L;
}

int resolve_path(const corr_ctx *c, int requested)
{
    if (requested != CORR_PATH_AUTO) return requested;
    if (tc_supported(c->n, c->device) && c->n >= 64) return CORR_PATH_TC_FP8;
    return CORR_PATH_CUDACORE;
}

bool path_supported(const corr_ctx *c, int path)
{
    switch (path) {
    case CORR_PATH_AUTO:
    case CORR_PATH_CUDACORE:
    case CORR_PATH_MMA_I8:
        return true;
    case CORR_PATH_TC_FP8:
        return tc_supported(c->n, c->device);
    default:
        return false;
    }
}

int cuda_fail(cudaError_t e)
{
    (void)e;
    return CORR_E_CUDA;
}

// Bracket a launch with timing events when profiling is on.
void prof_begin(corr_ctx *c, cudaStream_t s)
{
    if (!c->prof_on) return;
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (!c->prof_pool.empty()) {
        ev = c->prof_pool.back();
        c->prof_pool.pop_back();
    } else if (cudaEventCreate(&ev.first) != cudaSuccess ||
               cudaEventCreate(&ev.second) != cudaSuccess) {
        cudaGetLastError();
        c->prof_cur = {nullptr, nullptr};
        return;
    }
    cudaEventRecord(ev.first, s);
    c->prof_cur = ev;
}

void prof_end(corr_ctx *c, int kind, cudaStream_t s, int launches)
{
    c->prof_launches[kind] += launches;
    if (!c->prof_on || !c->prof_cur.first) return;
    cudaEventRecord(c->prof_cur.second, s);
    c->prof_pending[kind].push_back(c->prof_cur);
    c->prof_cur = {nullptr, nullptr};
}

// Work-item shape of the tensor-core path chosen by corr_set_tile.
TcItems tc_items(const corr_ctx *c)
{
    return c->tile == 128 ? TcItems::kSingle : c->tile == 256 ? TcItems::kPairs : TcItems::kAuto;
}

// Order `s` after a host dump that may still be reading the accumulators.
int wait_host_dump(corr_ctx *c, cudaStream_t s)
{
    if (!c->out_pending) return CORR_OK;
    if (cudaStreamWaitEvent(s, c->ev_out_free, 0) != cudaSuccess) {
        cudaGetLastError();
        return CORR_E_CUDA;
    }
    c->out_pending = false;
    return CORR_OK;
}

// Correlate n_time samples already in device memory into the packed triangle
// `target` (the context's accumulators, or a caller's output buffer for a
// whole integration); fresh: the first launch stores instead of adding.
// With `beam` set, the incoherent beam of the same samples goes to beam
// [nt / beam_avg][n_chan]: added by the tensor-core kernel's converters
// (the caller zeroes it first), written by the stand-alone beam kernel on the
// other paths.
int accumulate_to(corr_ctx *c, const uint8_t *volt, int nt, int32_t *target, bool fresh, cudaStream_t s,
                  int32_t *beam = nullptr, int beam_avg = 1)
{
    const int path = resolve_path(c, c->path);
    const bool zi = (c->flags & CORR_ZERO_INVALID) != 0;
    cudaError_t e = cudaSuccess;
    const size_t row = size_t(c->f) * size_t(c->n);
    if (path == CORR_PATH_TC_FP8) {
        // rows of n % 16 != 0 inputs go through a padded copy, chunk by chunk
        const int pad_t = tc_pad_samples(c->n, c->f, c->t_max);
        if (!pad_t && (reinterpret_cast<uintptr_t>(volt) & 15) != 0) return CORR_E_ARG;
        const int step = pad_t ? (pad_t < kTcMaxSamples ? pad_t : kTcMaxSamples) : kTcMaxSamples;
        for (int t0 = 0; t0 < nt; t0 += step) {
            const int ntc = nt - t0 < step ? nt - t0 : step;
            const uint8_t *src = volt + size_t(t0) * row;
            int ld = 0;
            if (pad_t) {
                prof_begin(c, s);
                e = launch_pad_rows(src, (long long)ntc * c->f, c->n, tc_ld(c->n), c->tc_pad, s);
                prof_end(c, CORR_K_UNPACK, s, 1);
                if (e != cudaSuccess) return cuda_fail(e);
                src = c->tc_pad;
                ld = tc_ld(c->n);
            }
            prof_begin(c, s);
            TcOptions opt;
            opt.wait_limit = c->wait_limit;
            opt.inject_stall = c->inject_stall;
            c->inject_stall = false;
            TcArray arr{src, target, c->f, c->n, ntc, zi, fresh, tc_items(c), ld};
            arr.beam = beam;
            arr.beam_avg = beam_avg;
            arr.beam_t0 = t0;
            e = launch_xeng_tc_batch(&arr, 1, c->status, opt, s);
            prof_end(c, CORR_K_XENGINE, s, 1);
            if (e != cudaSuccess) return cuda_fail(e);
            fresh = false;
        }
    } else if (path == CORR_PATH_CUDACORE) {
        const StagePlan &P = c->dp4a;
        const size_t plane_max = size_t(P.f_chunk) * (P.t_chunk / 2) * P.n_pad;
        int32_t *A = reinterpret_cast<int32_t *>(c->stage);
        int32_t *W = A + plane_max;
        const int tile = (c->tile == 32 || c->tile == 64) ? c->tile : (c->n <= 32 ? 32 : 64);
        const int n_pad = int(round_up(size_t(c->n), size_t(tile)));
        for (int t0 = 0; t0 < nt; t0 += P.t_chunk) {
            const int ntc = nt - t0 < P.t_chunk ? nt - t0 : P.t_chunk;
            const int tw_pad = int(round_up(size_t(ntc), 2 * kDp4aKW) / 2);
            for (int f0 = 0; f0 < c->f; f0 += P.f_chunk) {
                const int fc = c->f - f0 < P.f_chunk ? c->f - f0 : P.f_chunk;
                prof_begin(c, s);
                e = launch_unpack_words(volt + size_t(t0) * row, c->f, c->n, f0, fc, ntc, n_pad,
                                        tw_pad, zi, A, W, s);
                prof_end(c, CORR_K_UNPACK, s, 1);
                if (e != cudaSuccess) return cuda_fail(e);
                prof_begin(c, s);
                e = launch_xeng_dp4a(A, W, c->n, n_pad, fc, tw_pad, target, f0, fresh, tile, s);
                prof_end(c, CORR_K_XENGINE, s, 1);
                if (e != cudaSuccess) return cuda_fail(e);
            }
            fresh = false;
        }
    } else if (path == CORR_PATH_MMA_I8) {
        const StagePlan &P = c->mma;
        const size_t plane_max = size_t(P.f_chunk) * P.t_chunk * 2 * P.n_pad;
        int8_t *X = reinterpret_cast<int8_t *>(c->stage);
        int8_t *Xt = X + plane_max;
        for (int t0 = 0; t0 < nt; t0 += P.t_chunk) {
            const int ntc = nt - t0 < P.t_chunk ? nt - t0 : P.t_chunk;
            const int t_pad = int(round_up(size_t(ntc), kMmaKT));
            for (int f0 = 0; f0 < c->f; f0 += P.f_chunk) {
                const int fc = c->f - f0 < P.f_chunk ? c->f - f0 : P.f_chunk;
                prof_begin(c, s);
                e = launch_unpack_kmajor(volt + size_t(t0) * row, c->f, c->n, f0, fc, ntc, P.n_pad,
                                         t_pad, zi, X, Xt, s);
                prof_end(c, CORR_K_UNPACK, s, 1);
                if (e != cudaSuccess) return cuda_fail(e);
                prof_begin(c, s);
                e = launch_xeng_mma8(X, Xt, c->n, P.n_pad, fc, t_pad, target, f0, fresh, s);
                prof_end(c, CORR_K_XENGINE, s, 1);
                if (e != cudaSuccess) return cuda_fail(e);
            }
            fresh = false;
        }
    } else {
        return CORR_E_UNSUPPORTED;
    }
    if (beam && path != CORR_PATH_TC_FP8) {
        prof_begin(c, s);
        e = launch_beam(volt, nt, c->f, c->n, beam_avg, zi, beam, s);
        prof_end(c, CORR_K_OTHER, s, 1);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return CORR_OK;
}

// Add n_time samples to the running integration.
int accumulate_device(corr_ctx *c, const uint8_t *volt, int nt, cudaStream_t s)
{
    if (wait_host_dump(c, s) != CORR_OK) return CORR_E_CUDA;
    const int rc = accumulate_to(c, volt, nt, c->acc, c->fresh, s);
    if (rc != CORR_OK) return rc;
    c->fresh = false;
    return CORR_OK;
}

}  // namespace

namespace corr {

int set_last_error(int status) { return ret(status); }

StagePlan plan_dp4a(int n_inputs, int n_chan, int t_max)
{
    StagePlan P{};
    P.n_pad = int(round_up(size_t(n_inputs), kDp4aTile));
    size_t t_chunk = round_up(size_t(t_max), 2 * kDp4aKW);
    if (t_chunk > 8192) t_chunk = 8192;
    // two int32 planes of t_chunk/2 words per input: 4 * t_chunk * n_pad bytes/channel
    while (t_chunk > size_t(2 * kDp4aKW) && 4 * t_chunk * P.n_pad > kStageCap)
        t_chunk -= 2 * kDp4aKW;
    const size_t per_chan = 4 * t_chunk * P.n_pad;
    size_t fc = kStageCap / per_chan;
    if (fc < 1) fc = 1;
    if (fc > size_t(n_chan)) fc = size_t(n_chan);
    if (fc > 65535) fc = 65535;
    P.t_chunk = int(t_chunk);
    P.f_chunk = int(fc);
    P.bytes = per_chan * fc;
    return P;
}

StagePlan plan_mma(int n_inputs, int n_chan, int t_max)
{
    StagePlan P{};
    P.n_pad = int(round_up(size_t(n_inputs), kMmaTile));
    size_t t_chunk = round_up(size_t(t_max), kMmaKT);
    if (t_chunk > 8192) t_chunk = 8192;
    // two int8 planes (X and twisted) of 2 bytes per sample: 4 * t_chunk * n_pad bytes/channel
    while (t_chunk > size_t(kMmaKT) && 4 * t_chunk * P.n_pad > kStageCap) t_chunk -= kMmaKT;
    const size_t per_chan = 4 * t_chunk * P.n_pad;
    size_t fc = kStageCap / per_chan;
    if (fc < 1) fc = 1;
    if (fc > size_t(n_chan)) fc = size_t(n_chan);
    if (fc > 65535) fc = 65535;
    P.t_chunk = int(t_chunk);
    P.f_chunk = int(fc);
    P.bytes = per_chan * fc;
    return P;
}

}  // namespace corr

extern "C" {

corr_ctx *corr_create(int n_inputs, int n_chan, int n_time_per_int)
{
    if (n_inputs < 1 || n_chan < 1 || n_time_per_int < 1 || n_inputs > 8192 ||
        (long long)n_time_per_int * 128LL >= (1LL << 31)) {
        ret(CORR_E_ARG);
        return nullptr;
    }
    corr_ctx *c = new (std::nothrow) corr_ctx();
    if (!c) {
        ret(CORR_E_NOMEM);
        return nullptr;
    }
    c->n = n_inputs;
    c->f = n_chan;
    c->t_max = n_time_per_int;
    cudaDeviceProp prop;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        ret(CORR_E_CUDA);
        return nullptr;
    }
    c->sm_major = prop.major;
    c->sm_minor = prop.minor;
    c->sm_count = prop.multiProcessorCount;
    c->dp4a = plan_dp4a(n_inputs, n_chan, n_time_per_int);
    c->mma = plan_mma(n_inputs, n_chan, n_time_per_int);
    c->host_chunk = n_time_per_int < kHostChunk ? n_time_per_int : kHostChunk;
    if (cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->out_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_dumped, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_out_free, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        corr_destroy(c);
        ret(CORR_E_CUDA);
        return nullptr;
    }
    for (int b = 0; b < kHostBuffers; ++b) {
        if (cudaEventCreateWithFlags(&c->ev_full[b], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_free[b], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            corr_destroy(c);
            ret(CORR_E_CUDA);
            return nullptr;
        }
    }
    ret(CORR_OK);
    return c;
}

int corr_destroy(corr_ctx *c)
{
    if (!c) return ret(CORR_E_ARG);
    for (int b = 0; b < kHostBuffers; ++b) {
        if (c->ev_full[b]) cudaEventDestroy(c->ev_full[b]);
        if (c->ev_free[b]) cudaEventDestroy(c->ev_free[b]);
    }
    if (c->ev_dumped) cudaEventDestroy(c->ev_dumped);
    if (c->ev_out_free) cudaEventDestroy(c->ev_out_free);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->out_stream) cudaStreamDestroy(c->out_stream);
    for (int k = 0; k < CORR_K_KINDS; ++k)
        for (auto &ev : c->prof_pending[k]) c->prof_pool.push_back(ev);
    for (auto &ev : c->prof_pool) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    delete c;
    return ret(CORR_OK);
}

int corr_set_path(corr_ctx *c, int path)
{
    if (!c || path < CORR_PATH_AUTO || path > CORR_PATH_TC_FP8) return ret(CORR_E_ARG);
    if (c->samples != 0) return ret(CORR_E_STATE);
    if (!path_supported(c, path)) return ret(CORR_E_UNSUPPORTED);
    c->path = path;
    return ret(CORR_OK);
}

int corr_set_tile(corr_ctx *c, int tile)
{
    if (!c || (tile != 0 && tile != 32 && tile != 64 && tile != 128 && tile != 256)) return ret(CORR_E_ARG);
    if (c->samples != 0) return ret(CORR_E_STATE);
    c->tile = tile;
    return ret(CORR_OK);
}

int corr_set_wait_limit(corr_ctx *c, long long cycles)
{
    if (!c || cycles < 0) return ret(CORR_E_ARG);
    c->wait_limit = cycles;
    return ret(CORR_OK);
}

int corr_debug_inject(corr_ctx *c, unsigned what)
{
    if (!c || what > CORR_INJECT_STALL) return ret(CORR_E_ARG);
    c->inject_stall = what == CORR_INJECT_STALL;
    return ret(CORR_OK);
}

int corr_get_path(const corr_ctx *c)
{
    if (!c) return ret(CORR_E_ARG);
    g_last_error = CORR_OK;
    return resolve_path(c, c->path);
}

int corr_set_flags(corr_ctx *c, unsigned flags)
{
    if (!c || (flags & ~CORR_ZERO_INVALID)) return ret(CORR_E_ARG);
    if (c->samples != 0) return ret(CORR_E_STATE);
    c->flags = flags;
    return ret(CORR_OK);
}

size_t corr_workspace_bytes(const corr_ctx *c)
{
    if (!c) {
        ret(CORR_E_ARG);
        return 0;
    }
    g_last_error = CORR_OK;
    return layout_of(c).total;
}

size_t corr_workspace_bytes_for(int n_inputs, int n_chan, int n_time_per_int)
{
    if (n_inputs < 1 || n_chan < 1 || n_time_per_int < 1 || n_inputs > 8192 ||
        (long long)n_time_per_int * 128LL >= (1LL << 31)) {
        ret(CORR_E_ARG);
        return 0;
    }
    corr_ctx c;
    c.n = n_inputs;
    c.f = n_chan;
    c.t_max = n_time_per_int;
    c.dp4a = plan_dp4a(n_inputs, n_chan, n_time_per_int);
    c.mma = plan_mma(n_inputs, n_chan, n_time_per_int);
    c.host_chunk = n_time_per_int < kHostChunk ? n_time_per_int : kHostChunk;
    g_last_error = CORR_OK;
    return layout_of(&c).total;
}

int corr_bind_workspace(corr_ctx *c, void *d_ws, size_t bytes)
{
    if (!c || !d_ws || (reinterpret_cast<uintptr_t>(d_ws) % kAlign) != 0) return ret(CORR_E_ARG);
    const WsLayout L = layout_of(c);
    if (bytes < L.total) return ret(CORR_E_ARG);
    c->ws = static_cast<uint8_t *>(d_ws);
    c->ws_bytes = bytes;
    c->status = reinterpret_cast<DeviceStatus *>(c->ws + L.status_off);
    c->acc = reinterpret_cast<int32_t *>(c->ws + L.acc_off);
    c->stage = c->ws + L.stage_off;
    for (int b = 0; b < kHostBuffers; ++b) c->host_stage[b] = c->ws + L.host_off[b];
    c->tc_pad = c->ws + L.pad_off;
    c->host_next = 0;
    c->out_pending = false;
    c->samples = 0;
    c->fresh = true;
    if (cudaMemset(c->status, 0, sizeof(DeviceStatus)) != cudaSuccess) {
        cudaGetLastError();
        return ret(CORR_E_CUDA);
    }
    return ret(CORR_OK);
}

int corr_accumulate(corr_ctx *c, const uint8_t *d_volt, int n_time, void *stream)
{
    Range nvtx_range("corr_accumulate");
    if (!c || n_time < 0) return ret(CORR_E_ARG);
    if (!c->ws) return ret(CORR_E_STATE);
    if (n_time == 0) return ret(CORR_OK);
    if (!d_volt) return ret(CORR_E_ARG);
    if (c->samples + n_time > c->t_max) return ret(CORR_E_OVERFLOW);
    const int rc = accumulate_device(c, d_volt, n_time, static_cast<cudaStream_t>(stream));
    if (rc != CORR_OK) return ret(rc);
    c->samples += n_time;
    return ret(CORR_OK);
}

int corr_dump(corr_ctx *c, int32_t *d_vis, void *stream)
{
    Range nvtx_range("corr_dump");
    if (!c || !d_vis) return ret(CORR_E_ARG);
    if (!c->ws) return ret(CORR_E_STATE);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int launches = 0;
    prof_begin(c, s);
    cudaError_t e = launch_dump(c->acc, d_vis, acc_words(c), c->fresh, s, &launches);
    prof_end(c, CORR_K_DUMP, s, launches);
    if (e != cudaSuccess) return ret(cuda_fail(e));
    c->fresh = true;
    c->samples = 0;
    return ret(CORR_OK);
}

int corr_integrate(corr_ctx *c, const uint8_t *d_volt, int n_time, int32_t *d_vis, void *stream)
{
    Range nvtx_range("corr_integrate");
    if (!c || n_time < 0 || !d_vis) return ret(CORR_E_ARG);
    if (!c->ws) return ret(CORR_E_STATE);
    if (n_time > c->t_max) return ret(CORR_E_OVERFLOW);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n_time == 0) {
        if (cudaMemsetAsync(d_vis, 0, acc_words(c) * sizeof(int32_t), s) != cudaSuccess) {
            cudaGetLastError();
            return ret(CORR_E_CUDA);
        }
        return ret(CORR_OK);
    }
    if (!d_volt) return ret(CORR_E_ARG);
    return ret(accumulate_to(c, d_volt, n_time, d_vis, true, s));
}

int corr_integrate_beam(corr_ctx *c, const uint8_t *d_volt, int n_time, int32_t *d_vis, int32_t *d_beam,
                        int n_avg, void *stream)
{
    Range nvtx_range("corr_integrate_beam");
    if (!c || n_time < 0 || !d_vis || !d_beam || n_avg < 1 || n_time % n_avg != 0 ||
        (long long)n_avg * c->n * 128LL >= (1LL << 31))
        return ret(CORR_E_ARG);
    if (!c->ws) return ret(CORR_E_STATE);
    if (n_time > c->t_max) return ret(CORR_E_OVERFLOW);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n_time == 0) {
        if (cudaMemsetAsync(d_vis, 0, acc_words(c) * sizeof(int32_t), s) != cudaSuccess) {
            cudaGetLastError();
            return ret(CORR_E_CUDA);
        }
        return ret(CORR_OK);
    }
    if (!d_volt) return ret(CORR_E_ARG);
    if (resolve_path(c, c->path) == CORR_PATH_TC_FP8 &&
        cudaMemsetAsync(d_beam, 0, size_t(n_time / n_avg) * size_t(c->f) * sizeof(int32_t), s) != cudaSuccess) {
        cudaGetLastError();
        return ret(CORR_E_CUDA);
    }
    return ret(accumulate_to(c, d_volt, n_time, d_vis, true, s, d_beam, n_avg));
}

long long corr_samples(const corr_ctx *c)
{
    if (!c) {
        ret(CORR_E_ARG);
        return -1;
    }
    g_last_error = CORR_OK;
    return c->samples;
}

int corr_accumulate_host(corr_ctx *c, const uint8_t *h_volt, int n_time, void *stream)
{
    Range nvtx_range("corr_accumulate_host");
    if (!c || n_time < 0) return ret(CORR_E_ARG);
    if (!c->ws) return ret(CORR_E_STATE);
    if (n_time == 0) return ret(CORR_OK);
    if (!h_volt) return ret(CORR_E_ARG);
    if (c->samples + n_time > c->t_max) return ret(CORR_E_OVERFLOW);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t row = size_t(c->f) * size_t(c->n);
    for (int t0 = 0; t0 < n_time; t0 += c->host_chunk) {
        const int ntc = n_time - t0 < c->host_chunk ? n_time - t0 : c->host_chunk;
        const int b = c->host_next;
        c->host_next = (b + 1) % kHostBuffers;
        if (cudaStreamWaitEvent(c->copy_stream, c->ev_free[b], 0) != cudaSuccess ||
            cudaMemcpyAsync(c->host_stage[b], h_volt + size_t(t0) * row, size_t(ntc) * row,
                            cudaMemcpyHostToDevice, c->copy_stream) != cudaSuccess ||
            cudaEventRecord(c->ev_full[b], c->copy_stream) != cudaSuccess ||
            cudaStreamWaitEvent(s, c->ev_full[b], 0) != cudaSuccess) {
            cudaGetLastError();
            return ret(CORR_E_CUDA);
        }
        const int rc = accumulate_device(c, c->host_stage[b], ntc, s);
        if (rc != CORR_OK) return ret(rc);
        c->samples += ntc;
        if (cudaEventRecord(c->ev_free[b], s) != cudaSuccess) {
            cudaGetLastError();
            return ret(CORR_E_CUDA);
        }
    }
    return ret(CORR_OK);
}

int corr_dump_host(corr_ctx *c, int32_t *h_vis, void *stream)
{
    Range nvtx_range("corr_dump_host");
    if (!c || !h_vis) return ret(CORR_E_ARG);
    if (!c->ws) return ret(CORR_E_STATE);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = acc_words(c) * sizeof(int32_t);
    // a fresh context holds no data: zero the accumulators first, but only after
    // an earlier host dump's copy (on the output stream) has finished reading them
    if (c->fresh && wait_host_dump(c, s) != CORR_OK) return ret(CORR_E_CUDA);
    if (c->fresh && cudaMemsetAsync(c->acc, 0, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return ret(CORR_E_CUDA);
    }
    // the copy runs on the output stream, so the correlation work that follows
    // on `stream` (the next integration's host chunks) overlaps it; the next
    // write of the accumulators waits for it (out_pending)
    if (cudaEventRecord(c->ev_dumped, s) != cudaSuccess ||
        cudaStreamWaitEvent(c->out_stream, c->ev_dumped, 0) != cudaSuccess ||
        cudaMemcpyAsync(h_vis, c->acc, bytes, cudaMemcpyDeviceToHost, c->out_stream) != cudaSuccess ||
        cudaEventRecord(c->ev_out_free, c->out_stream) != cudaSuccess) {
        cudaGetLastError();
        return ret(CORR_E_CUDA);
    }
    c->out_pending = true;
    c->fresh = true;
    c->samples = 0;
    return ret(CORR_OK);
}

int corr_sync(corr_ctx *c, void *stream)
{
    if (!c) return ret(CORR_E_ARG);
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess ||
        (c->out_stream && cudaStreamSynchronize(c->out_stream) != cudaSuccess)) {
        cudaGetLastError();
        return ret(CORR_E_CUDA);
    }
    if (!c->status) return ret(CORR_OK);
    DeviceStatus st{};
    if (cudaMemcpy(&st, c->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return ret(CORR_E_CUDA);
    }
    if (st.code != 0) {
        cudaMemset(c->status, 0, sizeof(DeviceStatus));
        return ret(st.code);
    }
    return ret(CORR_OK);
}

struct StateHeader {
    uint32_t magic, version;
    int32_t n, f;
    int64_t samples;
    int64_t reserved;
};
static_assert(sizeof(StateHeader) == 32, "state header is 32 bytes");
static const uint32_t kStateMagic = 0x52524F43u;  // "CORR"

size_t corr_state_bytes(const corr_ctx *c)
{
    if (!c) {
        ret(CORR_E_ARG);
        return 0;
    }
    g_last_error = CORR_OK;
    return sizeof(StateHeader) + acc_words(c) * sizeof(int32_t);
}

int corr_get_state(corr_ctx *c, void *h_buf, size_t bytes, void *stream)
{
    if (!c || !h_buf || bytes < corr_state_bytes(c)) return ret(CORR_E_ARG);
    if (!c->ws) return ret(CORR_E_STATE);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StateHeader h{kStateMagic, 1u, c->n, c->f, c->samples, 0};
    std::memcpy(h_buf, &h, sizeof(h));
    uint8_t *dst = static_cast<uint8_t *>(h_buf) + sizeof(h);
    const size_t nb = acc_words(c) * sizeof(int32_t);
    if (c->fresh) {
        std::memset(dst, 0, nb);
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return ret(CORR_E_CUDA);
        }
        return ret(CORR_OK);
    }
    if (cudaMemcpyAsync(dst, c->acc, nb, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return ret(CORR_E_CUDA);
    }
    return ret(CORR_OK);
}

int corr_set_state(corr_ctx *c, const void *h_buf, size_t bytes, void *stream)
{
    if (!c || !h_buf || bytes < corr_state_bytes(c)) return ret(CORR_E_ARG);
    if (!c->ws) return ret(CORR_E_STATE);
    StateHeader h;
    std::memcpy(&h, h_buf, sizeof(h));
    if (h.magic != kStateMagic || h.version != 1u || h.n != c->n || h.f != c->f ||
        h.samples < 0 || h.samples > c->t_max)
        return ret(CORR_E_ARG);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint8_t *src = static_cast<const uint8_t *>(h_buf) + sizeof(h);
    const size_t nb = acc_words(c) * sizeof(int32_t);
    if (wait_host_dump(c, s) != CORR_OK) return ret(CORR_E_CUDA);
    if (cudaMemcpyAsync(c->acc, src, nb, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return ret(CORR_E_CUDA);
    }
    c->samples = h.samples;
    c->fresh = false;
    return ret(CORR_OK);
}

int corr_incoherent_beam(const uint8_t *d_volt, int n_time, int n_chan, int n_inputs, int n_avg,
                         unsigned flags, int32_t *d_beam, void *stream)
{
    Range nvtx_range("corr_incoherent_beam");
    if (n_time < 0 || n_chan < 1 || n_chan > (1 << 24) || n_inputs < 1 || n_inputs > 65536 || n_avg < 1 ||
        n_time % n_avg != 0 || (long long)n_avg * n_inputs * 128LL >= (1LL << 31) ||
        (flags & ~CORR_ZERO_INVALID))
        return ret(CORR_E_ARG);
    if (n_time == 0) return ret(CORR_OK);
    if (!d_volt || !d_beam) return ret(CORR_E_ARG);
    const cudaError_t e = launch_beam(d_volt, n_time, n_chan, n_inputs, n_avg, (flags & CORR_ZERO_INVALID) != 0,
                                      d_beam, static_cast<cudaStream_t>(stream));
    return ret(e == cudaSuccess ? CORR_OK : cuda_fail(e));
}

int corr_ingest_packets(const uint8_t *d_packets, long long n_packets, int bank, uint8_t *d_volt, void *d_seen,
                        int32_t *d_counters, void *stream)
{
    Range nvtx_range("corr_ingest_packets");
    if (n_packets < 0 || bank < 0 || bank > 31 || !d_volt || !d_seen || !d_counters ||
        (n_packets > 0 && !d_packets) || (reinterpret_cast<uintptr_t>(d_packets) & 3) != 0 ||
        (reinterpret_cast<uintptr_t>(d_volt) & 15) != 0 || (reinterpret_cast<uintptr_t>(d_seen) & 3) != 0 ||
        (reinterpret_cast<uintptr_t>(d_counters) & 3) != 0)
        return ret(CORR_E_ARG);
    const cudaError_t e = launch_ingest(d_packets, n_packets, bank, d_volt, d_seen, d_counters,
                                        static_cast<cudaStream_t>(stream));
    return ret(e == cudaSuccess ? CORR_OK : cuda_fail(e));
}

int corr_fine_pfb(const int8_t *d_x, int n_coarse, int n_inputs, long long n_samples, const float *d_window,
                  int n_taps, float scale, uint8_t *d_volt, float *d_spec, void *stream)
{
    Range nvtx_range("corr_fine_pfb");
    if (!d_x || !d_window || (!d_volt && !d_spec) || n_coarse < 1 || n_coarse > 65535 || n_inputs < 1 ||
        n_inputs > 65536 || n_taps < 1 || n_samples % CORR_PFB_POINTS != 0 ||
        n_samples < (long long)CORR_PFB_POINTS * n_taps || n_samples / CORR_PFB_POINTS >= (1LL << 31) ||
        !isfinite(scale) || (reinterpret_cast<uintptr_t>(d_x) & 7) != 0 ||
        (reinterpret_cast<uintptr_t>(d_window) & 15) != 0 || (reinterpret_cast<uintptr_t>(d_spec) & 7) != 0)
        return ret(CORR_E_ARG);
    if (n_taps != 1 && n_taps != 12) return ret(CORR_E_UNSUPPORTED);
    const cudaError_t e = launch_fine_pfb(d_x, n_coarse, n_inputs, n_samples, d_window, n_taps, scale, d_volt,
                                          d_spec, static_cast<cudaStream_t>(stream));
    return ret(e == cudaSuccess ? CORR_OK : cuda_fail(e));
}

int corr_remap(const int32_t *const *d_tri, int n_dumps, int n_inputs, int n_chan, int f_avg,
               const int32_t *d_nat_of_pfb, int32_t *d_out, void *stream)
{
    Range nvtx_range("corr_remap");
    if (!d_tri || !d_out || n_dumps < 1 || n_dumps > CORR_REMAP_MAX_DUMPS || n_inputs < 2 ||
        n_inputs % 2 != 0 || n_inputs > 8192 || n_chan < 1 || n_chan > 65535 || f_avg < 1 ||
        n_chan % f_avg != 0 || (!d_nat_of_pfb && n_inputs % 64 != 0))
        return ret(CORR_E_ARG);
    if ((reinterpret_cast<uintptr_t>(d_out) & 15) != 0) return ret(CORR_E_ARG);
    for (int d = 0; d < n_dumps; ++d)
        if (!d_tri[d] || (reinterpret_cast<uintptr_t>(d_tri[d]) & 7) != 0) return ret(CORR_E_ARG);
    const cudaError_t e = launch_remap(d_tri, n_dumps, n_inputs, n_chan, f_avg, d_nat_of_pfb, d_out,
                                       static_cast<cudaStream_t>(stream));
    return ret(e == cudaSuccess ? CORR_OK : cuda_fail(e));
}

int corr_unpack(const uint8_t *d_volt, int n_time, int n_chan, int n_inputs, int8_t *d_out,
                unsigned flags, void *stream)
{
    Range nvtx_range("corr_unpack");
    if (n_time < 0 || n_chan < 1 || n_inputs < 1 || n_chan > 65535 ||
        (flags & ~CORR_ZERO_INVALID))
        return ret(CORR_E_ARG);
    if (n_time == 0) return ret(CORR_OK);
    if (!d_volt || !d_out) return ret(CORR_E_ARG);
    cudaError_t e = launch_unpack_kmajor(d_volt, n_chan, n_inputs, 0, n_chan, n_time, n_inputs,
                                         n_time, (flags & CORR_ZERO_INVALID) != 0, d_out,
                                         nullptr, static_cast<cudaStream_t>(stream));
    return ret(e == cudaSuccess ? CORR_OK : CORR_E_CUDA);
}

/* ------------------------------------------------------------------- batch */

}  // extern "C"

struct corr_batch {
    int n = 0;
    corr_ctx *ctx[CORR_BATCH_MAX] = {};
    size_t ws_off[CORR_BATCH_MAX] = {};
    size_t ws_bytes[CORR_BATCH_MAX] = {};
    size_t total = 0;
    bool bound = false;
};

extern "C" {

corr_batch *corr_batch_create(int n_arrays, const corr_array_desc *descs)
{
    if (n_arrays < 1 || n_arrays > CORR_BATCH_MAX || !descs) {
        ret(CORR_E_ARG);
        return nullptr;
    }
    corr_batch *b = new (std::nothrow) corr_batch();
    if (!b) {
        ret(CORR_E_NOMEM);
        return nullptr;
    }
    for (int a = 0; a < n_arrays; ++a) {
        const corr_array_desc &d = descs[a];
        corr_ctx *c = corr_create(d.n_inputs, d.n_chan, d.n_time_per_int);
        int rc = c ? CORR_OK : corr_last_error();
        if (rc == CORR_OK) rc = corr_set_flags(c, d.flags);
        if (rc == CORR_OK) rc = corr_set_path(c, d.path);
        if (rc == CORR_OK) rc = corr_set_tile(c, d.tile);
        if (rc != CORR_OK) {
            if (c) corr_destroy(c);
            b->n = a;
            corr_batch_destroy(b);
            ret(rc);
            return nullptr;
        }
        b->ctx[a] = c;
        b->ws_off[a] = b->total;
        b->ws_bytes[a] = corr_workspace_bytes(c);
        b->total = round_up(b->total + b->ws_bytes[a], kAlign);
    }
    b->n = n_arrays;
    ret(CORR_OK);
    return b;
}

int corr_batch_destroy(corr_batch *b)
{
    if (!b) return ret(CORR_E_ARG);
    for (int a = 0; a < b->n; ++a)
        if (b->ctx[a]) corr_destroy(b->ctx[a]);
    delete b;
    return ret(CORR_OK);
}

size_t corr_batch_workspace_bytes(const corr_batch *b)
{
    if (!b) {
        ret(CORR_E_ARG);
        return 0;
    }
    g_last_error = CORR_OK;
    return b->total;
}

int corr_batch_bind_workspace(corr_batch *b, void *d_ws, size_t bytes)
{
    if (!b || !d_ws || (reinterpret_cast<uintptr_t>(d_ws) % kAlign) != 0 || bytes < b->total)
        return ret(CORR_E_ARG);
    for (int a = 0; a < b->n; ++a) {
        const int rc = corr_bind_workspace(b->ctx[a], static_cast<uint8_t *>(d_ws) + b->ws_off[a],
                                           b->ws_bytes[a]);
        if (rc != CORR_OK) return ret(rc);
    }
    b->bound = true;
    return ret(CORR_OK);
}

int corr_batch_path(const corr_batch *b, int a)
{
    if (!b || a < 0 || a >= b->n) return ret(CORR_E_ARG);
    return corr_get_path(b->ctx[a]);
}

long long corr_batch_samples(const corr_batch *b, int a)
{
    if (!b || a < 0 || a >= b->n) {
        ret(CORR_E_ARG);
        return -1;
    }
    return corr_samples(b->ctx[a]);
}

corr_ctx *corr_batch_array(corr_batch *b, int a)
{
    if (!b || a < 0 || a >= b->n) {
        ret(CORR_E_ARG);
        return nullptr;
    }
    g_last_error = CORR_OK;
    return b->ctx[a];
}

namespace {

// Correlate every array of a batch that has data: tensor-core arrays in one
// persistent launch per group of up to CORR_BATCH_TC_GROUP arrays and per
// kTcMaxSamples samples, the others on their own kernels.  With `into` null
// the samples are added to the arrays' running integrations; otherwise each
// array's whole integration is written to into[a] (its accumulators are left
// alone).
int batch_correlate(corr_batch *b, const uint8_t *const *d_volt, const int *n_time, int32_t *const *into,
                    cudaStream_t s)
{
    int tc[CORR_BATCH_MAX], n_tc = 0, max_nt = 0;
    for (int a = 0; a < b->n; ++a) {
        if (!d_volt[a] || n_time[a] == 0 || (into && !into[a])) continue;
        if (resolve_path(b->ctx[a], b->ctx[a]->path) == CORR_PATH_TC_FP8 && b->ctx[a]->n % 16 == 0) {
            tc[n_tc++] = a;
            if (n_time[a] > max_nt) max_nt = n_time[a];
        }
    }
    for (int g0 = 0; g0 < n_tc; g0 += CORR_BATCH_TC_GROUP) {
        const int gn = n_tc - g0 < CORR_BATCH_TC_GROUP ? n_tc - g0 : CORR_BATCH_TC_GROUP;
        corr_ctx *lead = b->ctx[tc[g0]];
        for (int x = 0; x < gn; ++x)
            if ((reinterpret_cast<uintptr_t>(d_volt[tc[g0 + x]]) & 15) != 0) return CORR_E_ARG;
        if (!into) {
            // the launch writes the arrays' accumulators: order it after any host
            // dump of them that may still be copying out on an output stream
            for (int x = 0; x < gn; ++x)
                if (wait_host_dump(b->ctx[tc[g0 + x]], s) != CORR_OK) return CORR_E_CUDA;
        }
        for (int t0 = 0; t0 < max_nt; t0 += kTcMaxSamples) {
            TcArray arr[CORR_BATCH_TC_GROUP];
            int k = 0;
            for (int x = 0; x < gn; ++x) {
                const int a = tc[g0 + x];
                corr_ctx *c = b->ctx[a];
                const int nt = n_time[a];
                const int ntc = nt - t0 <= 0 ? 0 : (nt - t0 < kTcMaxSamples ? nt - t0 : kTcMaxSamples);
                arr[k].volt = d_volt[a] + size_t(t0 > nt ? nt : t0) * size_t(c->f) * size_t(c->n);
                arr[k].acc = into ? into[a] : c->acc;
                arr[k].n_chan = c->f;
                arr[k].n = c->n;
                arr[k].nt = ntc;
                arr[k].zero_invalid = (c->flags & CORR_ZERO_INVALID) != 0;
                arr[k].fresh = t0 == 0 ? (into ? true : c->fresh) : false;
                arr[k].items = tc_items(c);
                ++k;
            }
            TcOptions opt;
            opt.wait_limit = lead->wait_limit;
            opt.inject_stall = lead->inject_stall;
            lead->inject_stall = false;
            prof_begin(lead, s);
            cudaError_t e = launch_xeng_tc_batch(arr, k, lead->status, opt, s);
            prof_end(lead, CORR_K_XENGINE, s, 1);
            if (e != cudaSuccess) return cuda_fail(e);
        }
        if (!into) {
            for (int x = 0; x < gn; ++x) {
                corr_ctx *c = b->ctx[tc[g0 + x]];
                c->fresh = false;
                c->samples += n_time[tc[g0 + x]];
            }
        }
    }
    for (int a = 0; a < b->n; ++a) {
        if (!d_volt[a] || n_time[a] == 0 || (into && !into[a])) continue;
        if (resolve_path(b->ctx[a], b->ctx[a]->path) == CORR_PATH_TC_FP8 && b->ctx[a]->n % 16 == 0) continue;
        if (into) {
            const int rc = accumulate_to(b->ctx[a], d_volt[a], n_time[a], into[a], true, s);
            if (rc != CORR_OK) return rc;
        } else {
            const int rc = accumulate_device(b->ctx[a], d_volt[a], n_time[a], s);
            if (rc != CORR_OK) return rc;
            b->ctx[a]->samples += n_time[a];
        }
    }
    return CORR_OK;
}

}  // namespace

int corr_batch_accumulate(corr_batch *b, const uint8_t *const *d_volt, const int *n_time,
                          void *stream)
{
    Range nvtx_range("corr_batch_accumulate");
    if (!b || !d_volt || !n_time) return ret(CORR_E_ARG);
    if (!b->bound) return ret(CORR_E_STATE);
    // every check before anything is enqueued
    for (int a = 0; a < b->n; ++a) {
        if (n_time[a] < 0) return ret(CORR_E_ARG);
        if (!d_volt[a] || n_time[a] == 0) continue;
        if (b->ctx[a]->samples + n_time[a] > b->ctx[a]->t_max) return ret(CORR_E_OVERFLOW);
    }
    return ret(batch_correlate(b, d_volt, n_time, nullptr, static_cast<cudaStream_t>(stream)));
}

int corr_batch_integrate(corr_batch *b, const uint8_t *const *d_volt, const int *n_time,
                         int32_t *const *d_vis, void *stream)
{
    Range nvtx_range("corr_batch_integrate");
    if (!b || !d_volt || !n_time || !d_vis) return ret(CORR_E_ARG);
    if (!b->bound) return ret(CORR_E_STATE);
    for (int a = 0; a < b->n; ++a) {
        if (n_time[a] < 0) return ret(CORR_E_ARG);
        if (!d_vis[a]) continue;
        if (n_time[a] > b->ctx[a]->t_max) return ret(CORR_E_OVERFLOW);
        if (n_time[a] > 0 && !d_volt[a]) return ret(CORR_E_ARG);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int a = 0; a < b->n; ++a) {
        if (!d_vis[a] || n_time[a] > 0) continue;
        if (cudaMemsetAsync(d_vis[a], 0, acc_words(b->ctx[a]) * sizeof(int32_t), s) != cudaSuccess) {
            cudaGetLastError();
            return ret(CORR_E_CUDA);
        }
    }
    return ret(batch_correlate(b, d_volt, n_time, d_vis, s));
}

int corr_batch_dump(corr_batch *b, int32_t *const *d_vis, void *stream)
{
    Range nvtx_range("corr_batch_dump");
    if (!b || !d_vis) return ret(CORR_E_ARG);
    if (!b->bound) return ret(CORR_E_STATE);
    for (int a = 0; a < b->n; ++a) {
        if (!d_vis[a]) continue;
        const int rc = corr_dump(b->ctx[a], d_vis[a], stream);
        if (rc != CORR_OK) return ret(rc);
    }
    return ret(CORR_OK);
}

int corr_batch_sync(corr_batch *b, void *stream)
{
    if (!b) return ret(CORR_E_ARG);
    int first = CORR_OK;
    for (int a = 0; a < b->n; ++a) {
        const int rc = corr_sync(b->ctx[a], stream);
        if (rc != CORR_OK && first == CORR_OK) first = rc;
    }
    return ret(first);
}

int corr_batch_graph_capture(corr_batch *b, const uint8_t *const *d_volt, const int *n_time,
                             int32_t *const *d_vis, void *stream, void **graph_exec)
{
    if (!b || !d_volt || !n_time || !d_vis || !graph_exec || !stream) return ret(CORR_E_ARG);
    if (!b->bound) return ret(CORR_E_STATE);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    *graph_exec = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return ret(CORR_E_CUDA);
    }
    // a whole integration straight into the output buffers: the accumulators
    // are not touched, so replays do not depend on the batch's state
    int rc = corr_batch_integrate(b, d_volt, n_time, d_vis, stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (rc != CORR_OK || e != cudaSuccess || !graph) {
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        return ret(rc != CORR_OK ? rc : CORR_E_CUDA);
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        return ret(CORR_E_CUDA);
    }
    *graph_exec = exec;
    return ret(CORR_OK);
}

int corr_graph_launch(void *graph_exec, void *stream)
{
    Range nvtx_range("corr_graph_launch");
    if (!graph_exec) return ret(CORR_E_ARG);
    if (cudaGraphLaunch(static_cast<cudaGraphExec_t>(graph_exec), static_cast<cudaStream_t>(stream)) !=
        cudaSuccess) {
        cudaGetLastError();
        return ret(CORR_E_CUDA);
    }
    return ret(CORR_OK);
}

int corr_graph_destroy(void *graph_exec)
{
    if (!graph_exec) return ret(CORR_E_ARG);
    cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(graph_exec));
    return ret(CORR_OK);
}

int corr_profile_enable(corr_ctx *c, int on)
{
    if (!c) return ret(CORR_E_ARG);
    c->prof_on = on != 0;
    return ret(CORR_OK);
}

int corr_profile_read(corr_ctx *c, corr_profile *out, int reset)
{
    if (!c || !out) return ret(CORR_E_ARG);
    for (int k = 0; k < CORR_K_KINDS; ++k) {
        double ms = 0.0;
        long long timed = 0;
        for (auto &ev : c->prof_pending[k]) {
            float t = 0.f;
            if (cudaEventSynchronize(ev.second) != cudaSuccess ||
                cudaEventElapsedTime(&t, ev.first, ev.second) != cudaSuccess) {
                cudaGetLastError();          // e.g. an event recorded inside a graph
                continue;
            }
            ms += t;
            ++timed;
        }
        out->launches[k] = c->prof_launches[k];
        out->timed[k] = timed;
        out->ms[k] = ms;
        if (reset) {
            for (auto &ev : c->prof_pending[k]) c->prof_pool.push_back(ev);
            c->prof_pending[k].clear();
            c->prof_launches[k] = 0;
        }
    }
    return ret(CORR_OK);
}

int corr_last_error(void) { return g_last_error; }

const char *corr_strerror(int status)
{
    switch (status) {
    case CORR_OK: return "success";
    case CORR_E_ARG: return "invalid argument";
    case CORR_E_STATE: return "call not valid in the current state";
    case CORR_E_OVERFLOW: return "integration would exceed n_time_per_int";
    case CORR_E_NOMEM: return "out of memory";
    case CORR_E_BUDGET: return "memory budget exceeded";
    case CORR_E_CUDA: return "CUDA runtime error";
    case CORR_E_TIMEOUT: return "device-side wait timed out";
    case CORR_E_UNSUPPORTED: return "unsupported shape or path on this device";
    default: return "unknown status";
    }
}

int corr_version(void) { return 100; }

}  // extern "C"
