// hs_serve.cu -- the serving form: a long-lived engine that admits requests
// into resident plane slots, produces each plane on the device (the stand-in
// for the upstream Fourier-domain stage), sums admitted groups with the
// batched kernels and returns every request's candidates to host memory.
//
// Threads: callers submit and wait; one dispatcher thread admits queued
// requests into free slots (memory admission), enqueues the group's plane
// generation, batched summing and result copies on the engine's stream and
// moves on to the next group at once (continuous batching: the GPU works
// through groups back to back while new requests arrive); one completion
// thread waits for each group's event in admission order, files the results
// and frees the slots.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include <cuda_bf16.h>

#include "hs_internal.h"

using namespace hs;

namespace {

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ----------------------
// Ten rounds of the published round function on a 128-bit counter with a
// 64-bit key bumped by the Weyl constants between rounds.
__host__ __device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    for (int i = 0; i < 10; ++i) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        c[1] = (uint32_t)p1;
        c[3] = (uint32_t)p0;
        c[0] = n0;
        c[2] = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// The ten round keys of a key (k0, k1): the same for every counter, so the
// noise kernel takes them as launch parameters instead of bumping the key
// in each thread.
struct RoundKeys {
    uint32_t k0[10], k1[10];
};

RoundKeys round_keys(uint32_t k0, uint32_t k1)
{
    RoundKeys r;
    for (int i = 0; i < 10; ++i) {
        r.k0[i] = k0;
        r.k1[i] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return r;
}

// philox4x32_10 with the round keys given.
__device__ __forceinline__ void philox4x32_10_rk(uint32_t c[4], const RoundKeys &rk)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ rk.k0[i];
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ rk.k1[i];
        c[1] = (uint32_t)p1;
        c[3] = (uint32_t)p0;
        c[0] = n0;
        c[2] = n2;
    }
}

constexpr uint32_t kNoiseTag = 0x6E6F6973u;  // counter word 3 of the noise stream
constexpr uint32_t kSignalTag = 0x7369676Eu; // counter word 3 of the signal draws
constexpr int kMaxSignals = 16;
constexpr int kSignalHarmonics = 16;

// Exponential(mean 1) from 32 random bits: u = (r + 1/2) 2^-32 in (0, 1],
// x = -ln u (at most ln 2^33 = 22.9, so tails used by thresholds of
// false-alarm rate 1e-8 still occur); 0 - ln u keeps x = +0 at u = 1.  The
// hardware logarithm (__logf) is accurate enough for a noise source and
// keeps the generator near the write bandwidth.
__device__ __forceinline__ float exp1(uint32_t r)
{
    const float u = fmaf((float)r, 2.3283064365386963e-10f, 1.1641532182693481e-10f);
    return fmaxf(0.0f - __logf(u), 0.0f);
}

// Noise plane, one Philox call per 4 consecutive bins of a row (grid.y =
// row).  A thread makes kQuadsPerThread quads, blockDim.x quads apart, so each
// store instruction of a warp writes contiguous bytes.
constexpr int kQuadsPerThread = 4;

template <bool LOWP>
__global__ void synth_noise(float *__restrict__ f32, __nv_bfloat16 *__restrict__ bf, long long n,
                            long long ld, long long width, const __grid_constant__ RoundKeys rk)
{
    const int row = (int)blockIdx.y;
    const long long quads = width / 4; // bins [0, width) of the row are written
    const long long q0 = (long long)blockIdx.x * blockDim.x * kQuadsPerThread + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kQuadsPerThread; ++k) {
        const long long q = q0 + (long long)k * blockDim.x;
        if (q >= quads)
            break;
        uint32_t c[4] = {(uint32_t)q, (uint32_t)(q >> 32), (uint32_t)row, kNoiseTag};
        philox4x32_10_rk(c, rk);
        const long long f = q * 4;
        float4 v;
        v.x = f + 0 < n ? exp1(c[0]) : 0.f;
        v.y = f + 1 < n ? exp1(c[1]) : 0.f;
        v.z = f + 2 < n ? exp1(c[2]) : 0.f;
        v.w = f + 3 < n ? exp1(c[3]) : 0.f;
        const long long at = (long long)row * ld + f;
        *reinterpret_cast<float4 *>(f32 + at) = v;
        if (LOWP) {
            __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y);
            __nv_bfloat162 hi = __floats2bfloat162_rn(v.z, v.w);
            uint2 w;
            w.x = *reinterpret_cast<uint32_t *>(&lo);
            w.y = *reinterpret_cast<uint32_t *>(&hi);
            *reinterpret_cast<uint2 *>(bf + at) = w;
        }
    }
}

struct SignalSet {
    int count;
    int z0[kMaxSignals];
    long long f0[kMaxSignals];
    float amp[kMaxSignals][kSignalHarmonics];
};

// Adds the signals in order on one thread, so overlapping harmonics add up
// the same way every time.
__global__ void synth_signals(float *f32, __nv_bfloat16 *bf, int n_templates, long long n,
                              long long ld, const __grid_constant__ SignalSet s)
{
    const int Z = (n_templates - 1) / 2;
    for (int i = 0; i < s.count; ++i)
        for (int h = 1; h <= kSignalHarmonics; ++h) {
            const long long f = h * s.f0[i];
            const int z = h * s.z0[i];
            if (f >= n || z > Z || z < -Z)
                continue;
            const long long at = (long long)(z + Z) * ld + f;
            const float v = f32[at] + s.amp[i][h - 1];
            f32[at] = v;
            if (bf)
                bf[at] = __float2bfloat16_rn(v);
        }
}

// Signal parameters drawn on the host from the seed: f0 uniform in
// [min(1e4, n/4), min(1e5, n/2)), z0 uniform in [-2, 2], amplitudes U[3, 8).
SignalSet draw_signals(uint64_t seed, long long n, int count)
{
    SignalSet s;
    std::memset(&s, 0, sizeof s);
    s.count = count;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    long long lo = std::min(10000LL, std::max(17LL, n / 4));
    long long hi = std::min(100000LL, std::max(lo + 1, n / 2));
    for (int i = 0; i < count; ++i) {
        uint32_t c[4] = {(uint32_t)i, 0u, 0u, kSignalTag};
        philox4x32_10(c, k0, k1);
        s.f0[i] = lo + (long long)(c[0] % (uint32_t)(hi - lo));
        s.z0[i] = (int)(c[1] % 5u) - 2;
        for (int j = 0; j < kSignalHarmonics / 4; ++j) {
            uint32_t d[4] = {(uint32_t)i, (uint32_t)(j + 1), 0u, kSignalTag};
            philox4x32_10(d, k0, k1);
            for (int t = 0; t < 4; ++t)
                s.amp[i][4 * j + t] = 3.0f + 5.0f * (float)(d[t] >> 8) * (1.0f / 16777216.0f);
        }
    }
    return s;
}

thread_local std::string g_err;

hs_status fail(hs_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

hs_status cuda_fail(cudaError_t e, const char *what)
{
    g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? HS_ERR_OOM : HS_ERR_CUDA;
}

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// write_pad: also zero the bins [n, ld) of every row (otherwise only the
// bins up to n rounded up to 4 are written).
hs_status synth(void *fop, float *fop32, int dtype, int nt, long long n, long long ld,
                uint64_t seed, int n_signals, cudaStream_t s, bool write_pad = true)
{
    if (!fop || reinterpret_cast<uintptr_t>(fop) % 16 != 0 || nt < 1 || n < 1 || ld < n ||
        ld % 8 != 0 || n_signals < 0 || n_signals > kMaxSignals ||
        (dtype != HS_F32 && dtype != HS_BF16))
        return fail(HS_ERR_INVALID, "hs_synth_fop: need a 16-byte aligned plane, 1 <= n_bins "
                                    "<= ld with ld a multiple of 8, dtype FP32 or BF16 and "
                                    "0..16 signals");
    if (dtype == HS_BF16 && (!fop32 || reinterpret_cast<uintptr_t>(fop32) % 16 != 0))
        return fail(HS_ERR_INVALID, "hs_synth_fop: a BF16 plane needs a 16-byte aligned FP32 copy");
    float *f32 = dtype == HS_F32 ? static_cast<float *>(fop) : fop32;
    __nv_bfloat16 *bf = dtype == HS_BF16 ? static_cast<__nv_bfloat16 *>(fop) : nullptr;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const long long width = write_pad ? ld : (n + 3) / 4 * 4;
    const long long quads = width / 4;
    const int tpb = 256;
    const long long per_block = (long long)tpb * kQuadsPerThread;
    const long long gx = (quads + per_block - 1) / per_block;
    if (gx > 0x7fffffffLL)
        return fail(HS_ERR_INVALID, "hs_synth_fop: row too long");
    const dim3 grid((unsigned)gx, (unsigned)nt);
    const RoundKeys rk = round_keys(k0, k1);
    if (bf)
        synth_noise<true><<<grid, tpb, 0, s>>>(f32, bf, n, ld, width, rk);
    else
        synth_noise<false><<<grid, tpb, 0, s>>>(f32, bf, n, ld, width, rk);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && n_signals > 0) {
        synth_signals<<<1, 1, 0, s>>>(f32, bf, nt, n, ld, draw_signals(seed, n, n_signals));
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? HS_OK : cuda_fail(e, "plane generator launch");
}

long long round8(long long x) { return (x + 7) / 8 * 8; }

struct Req {
    uint64_t ticket;
    hs_request r;
    int64_t t_submit, t_admit;
    int slot;
};

struct Group {
    std::vector<Req> reqs;
    int id = 0;
    int lane = 0; // stream index
    hs_status err = HS_OK;
    cudaEvent_t ev = nullptr;
};

struct Done {
    hs_result res;
    std::vector<hs_cand> recs;
};

} // namespace

struct hs_server {
    hs_server_config cfg{};
    std::vector<float> ta;
    int device = 0;
    long long ld_max = 0;
    float *d_f32 = nullptr;            // [n_slots][nt][ld_max] FP32 plane or FP32 copy
    __nv_bfloat16 *d_bf = nullptr;     // [n_slots][nt][ld_max] BF16 plane
    // per slot: 16 bytes of counters, then cand_capacity records; the
    // pinned host mirror has the same layout, so one copy returns a result
    unsigned char *d_out = nullptr;
    unsigned char *h_out = nullptr;
    size_t out_stride = 0;
    // per slot and dtype, the descriptors of the slot's plane (pitch ld_max)
    std::vector<StagedBatchBeam> slot_beam[2];
    // groups alternate between two streams, each with its own batches, so
    // one group's plane generation overlaps the previous group's summing
    static constexpr int kStreams = 2;
    cudaStream_t stream[kStreams] = {nullptr, nullptr};
    hs_batch *batch[kStreams][2] = {{nullptr, nullptr}, {nullptr, nullptr}}; // [stream][FP32, BF16]

    std::mutex mu;
    std::condition_variable cv_dispatch, cv_complete, cv_done;
    std::deque<Req> queue;
    std::deque<Group> inflight;
    std::vector<int> free_slots;
    std::vector<cudaEvent_t> events;
    std::unordered_map<uint64_t, Done> done;
    std::unordered_set<uint64_t> live;
    uint64_t next_ticket = 1;
    int n_groups = 0;
    int in_flight = 0;
    bool stop_dispatch = false, stop_complete = false;
    hs_server_stats st{};
    std::thread dispatcher, completer;
    int tile_order = 1; // linear: no per-group order table to build and upload
};

namespace {

uint32_t *slot_counters(unsigned char *base, size_t stride, int slot)
{
    return reinterpret_cast<uint32_t *>(base + stride * (size_t)slot);
}

hs_cand *slot_records(unsigned char *base, size_t stride, int slot)
{
    return reinterpret_cast<hs_cand *>(base + stride * (size_t)slot + 16);
}

void launch_group(hs_server *s, Group &g)
{
    const int nt = s->cfg.n_templates;
    const uint32_t cap = s->cfg.cand_capacity;
    const size_t slot_elems = (size_t)nt * (size_t)s->ld_max;
    cudaStream_t st_ = s->stream[g.lane];
    std::vector<StagedBatchBeam> beams[2];
    hs_status st = HS_OK;
    for (const Req &r : g.reqs) {
        const long long n = r.r.n_bins;
        const bool lowp = r.r.dtype == HS_BF16;
        StagedBatchBeam d;
        if (r.r.fop) { // resident plane: descriptors for the caller's memory
            std::memset(&d, 0, sizeof d);
            const long long ld = r.r.ld ? r.r.ld : n;
            const StagedShape sh{nt, s->cfg.H, 128, r.r.dtype};
            if (encode_plane_maps(sh, r.r.fop, n, ld, d.maps, d.split1) != CUDA_SUCCESS)
                st = fail(HS_ERR_CUDA, "cuTensorMapEncodeTiled failed for a resident plane");
            d.fop32 = lowp ? r.r.fop32 : nullptr;
            d.ld = ld;
        } else {
            float *f32 = s->d_f32 + slot_elems * r.slot;
            __nv_bfloat16 *bf = s->d_bf + slot_elems * r.slot;
            if (st == HS_OK)
                st = synth(lowp ? (void *)bf : (void *)f32, lowp ? f32 : nullptr, r.r.dtype, nt,
                           n, s->ld_max, r.r.seed, r.r.n_signals, st_, false);
            d = s->slot_beam[lowp ? 1 : 0][(size_t)r.slot];
            d.fop32 = lowp ? f32 : nullptr;
            d.ld = s->ld_max;
        }
        d.n = n;
        d.rec = slot_records(s->d_out, s->out_stride, r.slot);
        d.counters = slot_counters(s->d_out, s->out_stride, r.slot);
        d.cap = cap;
        d.tiles = (int)((n + 127) / 128);
        beams[lowp ? 1 : 0].push_back(d);
    }
    for (int d = 0; d < 2 && st == HS_OK; ++d) {
        if (beams[d].empty())
            continue;
        hs_batch *b = s->batch[g.lane][d];
        st = batch_set_prepared(b, beams[d].data(), (int)beams[d].size(), st_);
        if (st == HS_OK)
            st = hs_batch_run(b, reinterpret_cast<hs_stream_t>(st_));
        if (st != HS_OK)
            g_err = hs_batch_last_error();
    }
    cudaError_t e = cudaSuccess;
    for (const Req &r : g.reqs) {
        if (st != HS_OK || e != cudaSuccess)
            break;
        e = cudaMemcpyAsync(s->h_out + s->out_stride * r.slot, s->d_out + s->out_stride * r.slot,
                            s->out_stride, cudaMemcpyDeviceToHost, st_);
    }
    if (st == HS_OK && e == cudaSuccess)
        e = cudaEventRecord(g.ev, st_);
    if (st == HS_OK && e != cudaSuccess)
        st = cuda_fail(e, "serving group");
    g.err = st;
}

void dispatcher_main(hs_server *s)
{
    cudaSetDevice(s->device);
    const int max_group = s->cfg.max_group > 0 ? s->cfg.max_group : s->cfg.n_slots;
    for (;;) {
        Group g;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_dispatch.wait(lk, [&] {
                return s->stop_dispatch || (!s->queue.empty() && !s->free_slots.empty());
            });
            if (s->stop_dispatch)
                return;
            const int take = std::min({(int)s->queue.size(), (int)s->free_slots.size(), max_group});
            const int64_t t = now_ns();
            for (int i = 0; i < take; ++i) {
                Req r = s->queue.front();
                s->queue.pop_front();
                r.slot = s->free_slots.back();
                s->free_slots.pop_back();
                r.t_admit = t;
                g.reqs.push_back(r);
            }
            g.id = s->n_groups++;
            g.lane = g.id % hs_server::kStreams;
            s->in_flight += take;
            if (s->events.empty()) {
                g.ev = nullptr;
            } else {
                g.ev = s->events.back();
                s->events.pop_back();
            }
        }
        if (!g.ev && cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming |
                                                         cudaEventBlockingSync) != cudaSuccess) {
            g.ev = nullptr;
            g.err = HS_ERR_CUDA;
        } else {
            launch_group(s, g);
        }
        const int64_t t1 = now_ns();
        std::lock_guard<std::mutex> lk(s->mu);
        s->st.dispatch_ns += (uint64_t)(t1 - g.reqs.front().t_admit);
        s->inflight.push_back(std::move(g));
        s->st.groups++;
        s->cv_complete.notify_one();
    }
}

void completer_main(hs_server *s)
{
    cudaSetDevice(s->device);
    const uint32_t cap = s->cfg.cand_capacity;
    for (;;) {
        Group g;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_complete.wait(lk, [&] { return !s->inflight.empty() || s->stop_complete; });
            if (s->inflight.empty())
                return;
            g = std::move(s->inflight.front());
            s->inflight.pop_front();
        }
        hs_status gs = g.err;
        if (gs == HS_OK && cudaEventSynchronize(g.ev) != cudaSuccess)
            gs = HS_ERR_CUDA;
        const int64_t t = now_ns();
        std::vector<std::pair<uint64_t, Done>> out;
        out.reserve(g.reqs.size());
        uint64_t points = 0;
        for (const Req &r : g.reqs) {
            Done d;
            std::memset(&d.res, 0, sizeof d.res);
            d.res.ticket = r.ticket;
            d.res.group = g.id;
            d.res.group_size = (int32_t)g.reqs.size();
            d.res.slot = r.slot;
            d.res.t_submit_ns = r.t_submit;
            d.res.t_admit_ns = r.t_admit;
            d.res.t_done_ns = t;
            if (gs != HS_OK) {
                d.res.status = gs;
            } else {
                const uint32_t *c = slot_counters(s->h_out, s->out_stride, r.slot);
                const uint32_t cnt = c[0], dev = c[1];
                d.res.n_cands = cnt;
                d.res.status = dev != 0u ? (hs_status)dev : cnt > cap ? HS_ERR_OVERFLOW : HS_OK;
                const hs_cand *src = slot_records(s->h_out, s->out_stride, r.slot);
                d.recs.assign(src, src + std::min(cnt, cap));
                points += (uint64_t)s->cfg.n_templates * (uint64_t)r.r.n_bins;
            }
            out.emplace_back(r.ticket, std::move(d));
        }
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto &kv : out)
            s->done.emplace(kv.first, std::move(kv.second));
        for (const Req &r : g.reqs)
            s->free_slots.push_back(r.slot);
        if (g.ev)
            s->events.push_back(g.ev);
        s->in_flight -= (int)g.reqs.size();
        s->st.completed += g.reqs.size();
        s->st.points += points;
        s->cv_dispatch.notify_one();
        s->cv_done.notify_all();
    }
}

void free_server(hs_server *s)
{
    for (cudaStream_t st : s->stream)
        if (st)
            cudaStreamSynchronize(st);
    for (auto &lane : s->batch)
        for (hs_batch *b : lane)
            hs_batch_destroy(b);
    for (cudaEvent_t e : s->events)
        cudaEventDestroy(e);
    cudaFree(s->d_f32);
    cudaFree(s->d_bf);
    cudaFree(s->d_out);
    cudaFreeHost(s->h_out);
    for (cudaStream_t st : s->stream)
        if (st)
            cudaStreamDestroy(st);
    delete s;
}

} // namespace

extern "C" {

const char *hs_server_last_error(void) { return g_err.c_str(); }

hs_status hs_synth_fop(void *fop, float *fop32, int dtype, int n_templates, int64_t n_bins,
                       int64_t ld, uint64_t seed, int n_signals, hs_stream_t stream)
{
    return synth(fop, fop32, dtype, n_templates, n_bins, ld, seed, n_signals,
                 reinterpret_cast<cudaStream_t>(stream));
}

hs_status hs_server_create(hs_server **out, const hs_server_config *cfg)
{
    if (!out || !cfg)
        return fail(HS_ERR_INVALID, "out or cfg is null");
    *out = nullptr;
    const hs_server_config c = *cfg;
    if (c.n_templates < 1 || c.n_templates % 2 == 0 || c.H < 1 || !c.thresholds ||
        c.n_slots < 1 || c.n_slots > 1024 || c.slot_bins < 1 || c.slot_bins > 0x7fffffffLL ||
        c.cand_capacity < 1 || c.cand_capacity > (1u << 20) || c.queue_limit < 0 ||
        c.max_group < 0)
        return fail(HS_ERR_INVALID, "bad server configuration (odd n_templates, H >= 1, "
                                    "thresholds, 1..1024 slots, slot_bins >= 1, 1..2^20 "
                                    "records, queue_limit and max_group >= 0)");
    hs_server *s = new (std::nothrow) hs_server();
    if (!s)
        return fail(HS_ERR_OOM, "host allocation of the server failed");
    s->cfg = c;
    s->ta.assign(c.thresholds, c.thresholds + (size_t)c.H * c.n_templates);
    s->cfg.thresholds = s->ta.data();
    s->ld_max = round8(c.slot_bins);
    cudaGetDevice(&s->device);
    const int group = c.max_group > 0 ? c.max_group : c.n_slots;
    for (int l = 0; l < hs_server::kStreams; ++l)
        for (int d = 0; d < 2; ++d) {
            hs_options o{};
            o.dtype = d == 0 ? HS_F32 : HS_BF16;
            o.order = s->tile_order;
            o.assume_nonneg = c.assume_nonneg ? 1 : 0;
            const hs_status st = hs_batch_create(&s->batch[l][d], c.n_templates, c.H,
                                                 s->ta.data(), &o, group);
            if (st != HS_OK) {
                g_err = hs_batch_last_error();
                free_server(s);
                return st;
            }
        }
    const size_t elems = (size_t)c.n_slots * c.n_templates * (size_t)s->ld_max;
    cudaError_t e = cudaMalloc(&s->d_f32, elems * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&s->d_bf, elems * sizeof(__nv_bfloat16));
    s->out_stride = 16 + sizeof(hs_cand) * (size_t)c.cand_capacity;
    if (e == cudaSuccess)
        e = cudaMalloc(&s->d_out, s->out_stride * (size_t)c.n_slots);
    if (e == cudaSuccess)
        e = cudaMallocHost(&s->h_out, s->out_stride * (size_t)c.n_slots);
    for (int l = 0; l < hs_server::kStreams && e == cudaSuccess; ++l)
        e = cudaStreamCreateWithFlags(&s->stream[l], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        const hs_status st = cuda_fail(e, "reserving the server's slots");
        free_server(s);
        return st;
    }
    // descriptors of every slot's plane, encoded once: the plane of a
    // request of n bins keeps the slot's pitch, bins >= n are never summed
    const StagedShape sh32{c.n_templates, c.H, 128, HS_F32}, sh16{c.n_templates, c.H, 128, HS_BF16};
    for (int d = 0; d < 2; ++d)
        s->slot_beam[d].resize((size_t)c.n_slots);
    for (int i = 0; i < c.n_slots; ++i)
        for (int d = 0; d < 2; ++d) {
            StagedBatchBeam &b = s->slot_beam[d][(size_t)i];
            std::memset(&b, 0, sizeof b);
            const void *base = d == 0 ? (const void *)(s->d_f32 + (size_t)i * c.n_templates * s->ld_max)
                                      : (const void *)(s->d_bf + (size_t)i * c.n_templates * s->ld_max);
            if (encode_plane_maps(d == 0 ? sh32 : sh16, base, s->ld_max, s->ld_max, b.maps,
                                  b.split1) != CUDA_SUCCESS) {
                free_server(s);
                return fail(HS_ERR_CUDA, "cuTensorMapEncodeTiled failed for a slot");
            }
        }
    for (int i = c.n_slots - 1; i >= 0; --i)
        s->free_slots.push_back(i);
    s->st.free_slots = c.n_slots;
    try {
        s->dispatcher = std::thread(dispatcher_main, s);
        s->completer = std::thread(completer_main, s);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop_dispatch = s->stop_complete = true;
        }
        s->cv_dispatch.notify_all();
        s->cv_complete.notify_all();
        if (s->dispatcher.joinable())
            s->dispatcher.join();
        if (s->completer.joinable())
            s->completer.join();
        free_server(s);
        return fail(HS_ERR_OOM, "starting the server threads failed");
    }
    *out = s;
    return HS_OK;
}

hs_status hs_server_submit(hs_server *s, const hs_request *r, uint64_t *ticket)
{
    if (!s || !r || !ticket)
        return fail(HS_ERR_INVALID, "server, request or ticket is null");
    if (r->n_bins < 1 || r->n_bins > s->cfg.slot_bins || (r->dtype != HS_F32 &&
        r->dtype != HS_BF16) || r->n_signals < 0 || r->n_signals > kMaxSignals)
        return fail(HS_ERR_INVALID, "request needs 1 <= n_bins <= slot_bins, dtype FP32 or "
                                    "BF16 and 0..16 signals");
    if (r->fop) {
        const long long ld = r->ld ? r->ld : r->n_bins;
        const long long es = r->dtype == HS_F32 ? 4 : 2;
        if (reinterpret_cast<uintptr_t>(r->fop) % 16 != 0 || ld < r->n_bins ||
            (ld * es) % 16 != 0 ||
            (r->dtype == HS_BF16 &&
             (!r->fop32 || reinterpret_cast<uintptr_t>(r->fop32) % 16 != 0 || (ld * 4) % 16 != 0)))
            return fail(HS_ERR_INVALID, "resident plane: 16-byte aligned rows of pitch ld >= "
                                        "n_bins, and a BF16 plane's FP32 copy");
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.submitted++;
    // requests beyond the free slots wait; at most queue_limit of them
    if ((long long)s->queue.size() >= (long long)s->cfg.queue_limit + (long long)s->free_slots.size()) {
        s->st.rejected++;
        return fail(HS_ERR_BUSY, "queue full");
    }
    Req q;
    q.ticket = s->next_ticket++;
    q.r = *r;
    q.t_submit = now_ns();
    q.t_admit = 0;
    q.slot = -1;
    s->queue.push_back(q);
    s->live.insert(q.ticket);
    s->st.peak_queue = std::max(s->st.peak_queue, (int32_t)s->queue.size());
    *ticket = q.ticket;
    s->cv_dispatch.notify_one();
    return HS_OK;
}

hs_status hs_server_wait(hs_server *s, uint64_t ticket, int timeout_ms, hs_result *res,
                         hs_cand *records, uint32_t capacity)
{
    if (!s || !res)
        return fail(HS_ERR_INVALID, "server or result is null");
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->live.count(ticket))
        return fail(HS_ERR_INVALID, "unknown ticket");
    auto ready = [&] { return s->done.count(ticket) != 0; };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return fail(HS_ERR_BUSY, "request not finished");
    auto it = s->done.find(ticket);
    *res = it->second.res;
    if (records) {
        const size_t k = std::min(it->second.recs.size(), (size_t)capacity);
        std::copy(it->second.recs.begin(), it->second.recs.begin() + (long)k, records);
    }
    s->done.erase(it);
    s->live.erase(ticket);
    return HS_OK;
}

hs_status hs_server_drain(hs_server *s, int timeout_ms)
{
    if (!s)
        return fail(HS_ERR_INVALID, "server is null");
    std::unique_lock<std::mutex> lk(s->mu);
    auto idle = [&] { return s->queue.empty() && s->in_flight == 0; };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, idle);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle))
        return fail(HS_ERR_BUSY, "server still busy");
    return HS_OK;
}

hs_status hs_server_stats_get(hs_server *s, hs_server_stats *st)
{
    if (!s || !st)
        return fail(HS_ERR_INVALID, "server or stats is null");
    std::lock_guard<std::mutex> lk(s->mu);
    *st = s->st;
    st->queued = (int32_t)s->queue.size();
    st->in_flight = s->in_flight;
    st->free_slots = (int32_t)s->free_slots.size();
    return HS_OK;
}

hs_status hs_server_destroy(hs_server *s)
{
    if (!s)
        return HS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop_dispatch = true;
    }
    s->cv_dispatch.notify_all();
    if (s->dispatcher.joinable())
        s->dispatcher.join();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop_complete = true;
    }
    s->cv_complete.notify_all();
    if (s->completer.joinable())
        s->completer.join();
    free_server(s);
    return HS_OK;
}

} // extern "C"
