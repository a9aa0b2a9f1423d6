// hs_batch.cu -- the batched form: many planes (beams) of one shape.
// hs_batch_set_beams takes beams anywhere in device memory, each of its own
// length and row pitch, summed by a few launches that each carry up to K
// beams' TMA descriptors in their parameter block (K = 13 for the 85 x 16
// shape).  hs_batch_set_packed takes beams side by side along the bins of one
// plane: one set of descriptors serves them all and one launch sums every
// tile of every beam, reading the beam table and the (beam, tile) run order
// from device memory.  hs_batch_run launches; hs_batch_graph_run replays a
// CUDA graph of the same launches, captured again after the beams change.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "hs_internal.h"

using namespace hs;

struct hs_batch {
    int nt = 0, H = 0, dtype = HS_F32, tb = 128, order = 2;
    int max_beams = 0, total_tiles = 0;
    float delta = 0.f, band_abs = 0.f;
    std::vector<float> ta;
    float tmin[kMaxGroups];
    float *d_ta = nullptr;
    std::vector<StagedBatchBeam> beams;
    uint32_t *d_order = nullptr; // tile order of each beam, concatenated
    long long order_cap = 0;
    std::vector<uint32_t> h_order;
    std::vector<uint32_t> order_full; // order of the largest beam seen (a filter gives smaller ones)
    int grid_per_sm = 0;         // 0: one CTA per tile
    bool assume_nonneg = false;  // planes declared non-negative: no sign check
    int sms = 0;
    int device = 0;              // the device current at creation: its tables live there
    std::mutex mu;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_stale = true;     // beams changed since the graph was captured
    // packed batch (hs_batch_set_packed): one plane, one set of descriptors
    bool packed = false;
    CUtensorMap pmaps[kMaxStagedH];
    CUtensorMap psplit1[2];
    const float *pfop32 = nullptr;
    long long pitch = 0;
    PackedBeam *d_pbeams = nullptr;
    int pbeams_cap = 0, n_pbeams = 0;
    uint2 *d_ptiles = nullptr;
    long long ptiles_cap = 0;
    int n_ptiles = 0;
    std::vector<uint2> h_ptiles;
    std::vector<PackedBeam> h_pbeams;
};

namespace {

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

size_t elem_size(int dtype) { return dtype == HS_F32 ? 4 : 2; }

// A batch's tables live on the device that was current when it was made; a
// kernel launched with another device current would read them from there.
hs_status check_device(const hs_batch *b)
{
    int dev = -1;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    if (dev != b->device)
        return fail(HS_ERR_INVALID, "the batch belongs to another device: make that device "
                                    "current before using it");
    return HS_OK;
}

StagedBatch launch_args(const hs_batch *b)
{
    StagedBatch a{};
    a.sh = StagedShape{b->nt, b->H, b->tb, b->dtype};
    a.tmin_host = b->tmin;
    a.ta = b->d_ta;
    a.delta = b->delta;
    a.band_abs = b->band_abs;
    a.beams = b->beams.data();
    a.n_beams = (int)b->beams.size();
    a.order = b->order == 1 ? nullptr : b->d_order;
    a.grid_per_sm = b->grid_per_sm;
    a.sms = b->sms;
    a.assume_nonneg = b->assume_nonneg;
    return a;
}

PackedBatch packed_args(const hs_batch *b)
{
    PackedBatch a{};
    a.sh = StagedShape{b->nt, b->H, b->tb, b->dtype};
    a.maps = b->pmaps;
    a.split1 = b->psplit1;
    a.tmin_host = b->tmin;
    a.ta = b->d_ta;
    a.fop32 = b->pfop32;
    a.tiles = b->d_ptiles;
    a.beams = b->d_pbeams;
    a.n_beams = b->n_pbeams;
    a.n_tiles = b->n_ptiles;
    a.ld = b->pitch;
    a.delta = b->delta;
    a.band_abs = b->band_abs;
    a.grid_per_sm = b->grid_per_sm;
    a.sms = b->sms;
    a.assume_nonneg = b->assume_nonneg;
    return a;
}

// The launches of one run of the current beam set (on stream s).
cudaError_t launch_run(const hs_batch *b, cudaStream_t s)
{
    return b->packed ? launch_packed_batch(packed_args(b), s)
                     : launch_staged_batch(launch_args(b), s);
}

} // namespace

extern "C" {

const char *hs_batch_last_error(void) { return g_err.c_str(); }

hs_status hs_batch_create(hs_batch **out, int n_templates, int H, const float *thresholds,
                          const hs_options *opt, int max_beams)
{
    if (!out)
        return fail(HS_ERR_INVALID, "out is null");
    *out = nullptr;
    hs_options o{};
    if (opt)
        o = *opt;
    if (n_templates < 1 || n_templates % 2 == 0 || n_templates > 32767 || H < 1 || H > 32)
        return fail(HS_ERR_INVALID, "n_templates must be odd (1..32767) and H in [1, 32]");
    if (max_beams < 1 || max_beams > (1 << 16))
        return fail(HS_ERR_INVALID, "max_beams must be in [1, 65536]");
    if (!thresholds)
        return fail(HS_ERR_INVALID, "thresholds is null");
    for (long long i = 0; i < (long long)H * n_templates; ++i)
        if (!std::isfinite(thresholds[i]))
            return fail(HS_ERR_INVALID, "thresholds must be finite");
    if (o.dtype < HS_F32 || o.dtype > HS_F16 || o.grid_per_sm < 0 || o.grid_per_sm > 64 ||
        o.order < 0 || o.order > 4 || o.assume_nonneg < 0 || o.assume_nonneg > 1)
        return fail(HS_ERR_INVALID, "unknown option value");
    const StagedShape sh{n_templates, H, 128, o.dtype};
    if (!staged_batch_available(sh) || o.index != HS_INDEX_STRETCH ||
        o.zround != HS_ZROUND_SYMMETRIC)
        return fail(HS_ERR_UNSUPPORTED, "no batched kernel for this shape/options (compiled: "
                                        "85x16 FP32/BF16 and 21x8 FP32, stretch, symmetric)");
    hs_batch *b = new (std::nothrow) hs_batch();
    if (!b)
        return fail(HS_ERR_OOM, "host allocation of the batch failed");
    b->nt = n_templates;
    b->H = H;
    b->dtype = o.dtype;
    b->order = o.order == 0 ? 4 : o.order; // default: 53 steps to the octave
    b->assume_nonneg = o.assume_nonneg != 0;
    b->max_beams = max_beams;
    b->ta.assign(thresholds, thresholds + (size_t)H * n_templates);
    storage_error(b->dtype, H, &b->delta, &b->band_abs);
    group_bounds(b->ta.data(), n_templates, H, b->delta, b->band_abs, b->tmin);
    int dev = 0;
    cudaGetDevice(&dev);
    b->device = dev;
    cudaError_t e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    b->grid_per_sm = o.grid_per_sm;
    if (e == cudaSuccess)
        e = cudaMalloc(&b->d_ta, sizeof(float) * b->ta.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_ta, b->ta.data(), sizeof(float) * b->ta.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        hs_batch_destroy(b);
        return cuda_fail(e, "batch device tables");
    }
    *out = b;
    return HS_OK;
}

} // extern "C"

hs_status hs::batch_set_prepared(hs_batch *b, const StagedBatchBeam *beams, int n_beams,
                                 cudaStream_t s)
{
    if (n_beams < 0 || n_beams > b->max_beams)
        return fail(HS_ERR_INVALID, "n_beams must be in [0, max_beams]");
    std::vector<StagedBatchBeam> nb(beams, beams + n_beams);
    long long total = 0;
    for (const StagedBatchBeam &d : nb)
        total += d.tiles;
    if (total > 0x7fffffffLL)
        return fail(HS_ERR_INVALID, "batch has more than 2^31 tiles");
    std::lock_guard<std::mutex> lk(b->mu);
    cudaError_t e = cudaSuccess;
    if (b->order != 1) {
        // the order of t < k tiles is the order of more tiles
        // with the entries >= k dropped (the sort key depends on t alone)
        int most = 0;
        for (const StagedBatchBeam &d : nb)
            most = std::max(most, d.tiles);
        if ((int)b->order_full.size() < most)
            b->order_full = tile_order(most, b->order);
        b->h_order.resize((size_t)total);
        size_t at = 0;
        for (const StagedBatchBeam &d : nb) {
            if ((int)b->order_full.size() == d.tiles) {
                std::copy(b->order_full.begin(), b->order_full.end(), b->h_order.begin() + (long)at);
                at += (size_t)d.tiles;
            } else {
                for (uint32_t t : b->order_full)
                    if ((int)t < d.tiles)
                        b->h_order[at++] = t;
            }
        }
        if (total > b->order_cap) {
            // the old table may still be read by queued runs: wait for them
            e = cudaStreamSynchronize(s);
            if (e == cudaSuccess) {
                cudaFree(b->d_order);
                b->d_order = nullptr;
                b->order_cap = 0;
                e = cudaMalloc(&b->d_order, sizeof(uint32_t) * (size_t)total);
            }
            if (e != cudaSuccess)
                return cuda_fail(e, "allocating the tile order table");
            b->order_cap = total;
        }
        // pageable source: the copy completes its host-side read before return
        if (total > 0)
            e = cudaMemcpyAsync(b->d_order, b->h_order.data(), sizeof(uint32_t) * (size_t)total,
                                cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess)
            return cuda_fail(e, "uploading the tile order");
    }
    b->beams.swap(nb);
    b->total_tiles = (int)total;
    b->packed = false;
    b->graph_stale = true;
    return HS_OK;
}

extern "C" {

hs_status hs_batch_set_beams(hs_batch *b, const hs_beam *beams, int n_beams, hs_stream_t stream)
{
    if (!b || (!beams && n_beams > 0))
        return fail(HS_ERR_INVALID, "batch or beams is null");
    if (hs_status d = check_device(b); d != HS_OK)
        return d;
    if (n_beams < 0 || n_beams > b->max_beams)
        return fail(HS_ERR_INVALID, "n_beams must be in [0, max_beams]");
    const size_t es = elem_size(b->dtype);
    const StagedShape sh{b->nt, b->H, b->tb, b->dtype};
    std::vector<StagedBatchBeam> nb((size_t)n_beams);
    long long total = 0;
    for (int i = 0; i < n_beams; ++i) {
        const hs_beam &bm = beams[i];
        const long long ld = bm.ld ? bm.ld : bm.n_bins;
        if (!bm.fop || reinterpret_cast<uintptr_t>(bm.fop) % 16 != 0 || bm.n_bins < 1 ||
            bm.n_bins > 0x7fffffffLL || ld < bm.n_bins || (ld * (long long)es) % 16 != 0)
            return fail(HS_ERR_INVALID, "beam " + std::to_string(i) +
                                            ": plane must be 16-byte aligned with a row pitch "
                                            ">= n_bins and a multiple of 16 bytes");
        if (!bm.cands.count || (bm.cands.capacity > 0 && !bm.cands.records) ||
            reinterpret_cast<uintptr_t>(bm.cands.records) % 16 != 0)
            return fail(HS_ERR_INVALID, "beam " + std::to_string(i) + ": bad candidate buffer");
        if (bm.fop32 && (b->dtype == HS_F32 || reinterpret_cast<uintptr_t>(bm.fop32) % 16 != 0))
            return fail(HS_ERR_INVALID, "beam " + std::to_string(i) + ": bad FP32 copy");
        StagedBatchBeam &d = nb[(size_t)i];
        std::memset(&d, 0, sizeof d);
        if (encode_plane_maps(sh, bm.fop, bm.n_bins, ld, d.maps, d.split1) != CUDA_SUCCESS)
            return fail(HS_ERR_CUDA, "cuTensorMapEncodeTiled failed for beam " + std::to_string(i));
        d.fop32 = bm.fop32;
        d.n = bm.n_bins;
        d.ld = ld;
        d.rec = bm.cands.records;
        d.counters = bm.cands.count;
        d.cap = bm.cands.capacity;
        d.tiles = (int)((bm.n_bins + b->tb - 1) / b->tb);
        total += d.tiles;
        if (total > 0x7fffffffLL)
            return fail(HS_ERR_INVALID, "batch has more than 2^31 tiles");
    }
    return batch_set_prepared(b, nb.data(), n_beams, reinterpret_cast<cudaStream_t>(stream));
}

hs_status hs_batch_set_packed(hs_batch *b, const void *plane, const float *fop32, int64_t pitch,
                              const hs_packed_beam *beams, int n_beams, hs_stream_t stream)
{
    if (!b || (!beams && n_beams > 0))
        return fail(HS_ERR_INVALID, "batch or beams is null");
    if (hs_status d = check_device(b); d != HS_OK)
        return d;
    if (n_beams < 0 || n_beams > b->max_beams)
        return fail(HS_ERR_INVALID, "n_beams must be in [0, max_beams]");
    const long long es = (long long)elem_size(b->dtype);
    if (!plane || reinterpret_cast<uintptr_t>(plane) % 16 != 0 || pitch < 1 ||
        pitch > 0x7fffffffLL || (pitch * es) % 16 != 0)
        return fail(HS_ERR_INVALID, "packed plane must be 16-byte aligned with a pitch in "
                                    "[1, 2^31) that is a multiple of 16 bytes");
    if (fop32 && (b->dtype == HS_F32 || reinterpret_cast<uintptr_t>(fop32) % 16 != 0))
        return fail(HS_ERR_INVALID, "bad FP32 copy (16-bit batches only; 16-byte aligned)");
    const StagedShape sh{b->nt, b->H, b->tb, b->dtype};
    std::vector<PackedBeam> pb((size_t)n_beams);
    long long total = 0;
    int most = 0;
    for (int i = 0; i < n_beams; ++i) {
        const hs_packed_beam &bm = beams[i];
        if (bm.offset < 0 || bm.n_bins < 1 || bm.offset + bm.n_bins > pitch ||
            (bm.offset * es) % 16 != 0)
            return fail(HS_ERR_INVALID, "packed beam " + std::to_string(i) +
                                            ": need offset >= 0 a multiple of 16 bytes, "
                                            "n_bins >= 1, offset + n_bins <= pitch");
        if (!bm.cands.count || (bm.cands.capacity > 0 && !bm.cands.records) ||
            reinterpret_cast<uintptr_t>(bm.cands.records) % 16 != 0)
            return fail(HS_ERR_INVALID, "packed beam " + std::to_string(i) +
                                            ": bad candidate buffer");
        PackedBeam &d = pb[(size_t)i];
        std::memset(&d, 0, sizeof d);
        d.off = bm.offset;
        d.n = bm.n_bins;
        d.rec = bm.cands.records;
        d.counters = bm.cands.count;
        d.cap = bm.cands.capacity;
        const long long tiles = (bm.n_bins + b->tb - 1) / b->tb;
        total += tiles;
        most = std::max(most, (int)tiles);
        if (total > 0x7fffffffLL)
            return fail(HS_ERR_INVALID, "batch has more than 2^31 tiles");
    }
    CUtensorMap maps[kMaxStagedH], split1[2];
    if (encode_plane_maps(sh, plane, pitch, pitch, maps, split1) != CUDA_SUCCESS)
        return fail(HS_ERR_CUDA, "cuTensorMapEncodeTiled failed for the packed plane");
    // run order: each beam's tiles in the batch's tile order, beam after beam
    std::lock_guard<std::mutex> lk(b->mu);
    std::vector<uint2> tiles((size_t)total);
    {
        const std::vector<uint32_t> full =
            b->order == 1 ? std::vector<uint32_t>() : tile_order(most, b->order);
        size_t at = 0;
        for (int i = 0; i < n_beams; ++i) {
            const int t_b = (int)((pb[(size_t)i].n + b->tb - 1) / b->tb);
            if (b->order == 1) {
                for (int t = 0; t < t_b; ++t)
                    tiles[at++] = make_uint2((unsigned)i, (unsigned)t);
            } else {
                // the order of fewer tiles is the longer order with the
                // larger entries dropped (its sort key depends on t alone)
                for (uint32_t t : full)
                    if ((int)t < t_b)
                        tiles[at++] = make_uint2((unsigned)i, t);
            }
        }
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (n_beams > b->pbeams_cap || total > b->ptiles_cap) {
        // the old tables may still be read by queued runs: wait for them
        e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && n_beams > b->pbeams_cap) {
            cudaFree(b->d_pbeams);
            b->d_pbeams = nullptr;
            b->pbeams_cap = 0;
            e = cudaMalloc(&b->d_pbeams, sizeof(PackedBeam) * (size_t)n_beams);
            if (e == cudaSuccess)
                b->pbeams_cap = n_beams;
        }
        if (e == cudaSuccess && total > b->ptiles_cap) {
            cudaFree(b->d_ptiles);
            b->d_ptiles = nullptr;
            b->ptiles_cap = 0;
            e = cudaMalloc(&b->d_ptiles, sizeof(uint2) * (size_t)total);
            if (e == cudaSuccess)
                b->ptiles_cap = total;
        }
        if (e != cudaSuccess)
            return cuda_fail(e, "allocating the packed batch tables");
    }
    // copies from host memory this call owns until they have been read: the
    // vectors move into the batch, which keeps them until the next set
    b->h_pbeams.swap(pb);
    b->h_ptiles.swap(tiles);
    if (n_beams > 0)
        e = cudaMemcpyAsync(b->d_pbeams, b->h_pbeams.data(), sizeof(PackedBeam) * (size_t)n_beams,
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && total > 0)
        e = cudaMemcpyAsync(b->d_ptiles, b->h_ptiles.data(), sizeof(uint2) * (size_t)total,
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s); // the host tables may change at the next set
    if (e != cudaSuccess)
        return cuda_fail(e, "uploading the packed batch tables");
    std::memcpy(b->pmaps, maps, sizeof maps);
    std::memcpy(b->psplit1, split1, sizeof split1);
    b->pfop32 = fop32;
    b->pitch = pitch;
    b->n_pbeams = n_beams;
    b->n_ptiles = (int)total;
    b->total_tiles = (int)total;
    b->packed = true;
    b->graph_stale = true;
    return HS_OK;
}

hs_status hs_batch_run(hs_batch *b, hs_stream_t stream)
{
    if (!b)
        return fail(HS_ERR_INVALID, "batch is null");
    if (hs_status d = check_device(b); d != HS_OK)
        return d;
    std::lock_guard<std::mutex> lk(b->mu);
    cudaError_t e = launch_run(b, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? HS_OK : cuda_fail(e, "batched kernel launch");
}

hs_status hs_batch_graph_run(hs_batch *b, hs_stream_t stream)
{
    if (!b)
        return fail(HS_ERR_INVALID, "batch is null");
    if (hs_status d = check_device(b); d != HS_OK)
        return d;
    std::lock_guard<std::mutex> lk(b->mu);
    cudaError_t e = cudaSuccess;
    if (b->graph_stale || !b->gexec) {
        // capture the counter reset and the launches of the current beams;
        // update the instantiated graph in place when its topology allows
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t el = launch_run(b, b->cap_stream);
            e = cudaStreamEndCapture(b->cap_stream, &graph);
            if (e == cudaSuccess)
                e = el;
        }
        if (e == cudaSuccess && b->gexec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(b->gexec, graph, &info) != cudaSuccess) {
                cudaGetLastError(); // clear the update failure
                cudaGraphExecDestroy(b->gexec);
                b->gexec = nullptr;
            }
        }
        if (e == cudaSuccess && !b->gexec)
            e = cudaGraphInstantiate(&b->gexec, graph, 0);
        if (graph)
            cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->gexec = nullptr;
            return cuda_fail(e, "capturing the batch graph");
        }
        b->graph_stale = false;
    }
    e = cudaGraphLaunch(b->gexec, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? HS_OK : cuda_fail(e, "cudaGraphLaunch");
}

int hs_batch_tiles(const hs_batch *b) { return b ? b->total_tiles : 0; }

int hs_batch_launches(const hs_batch *b)
{
    if (!b)
        return 0;
    if (b->packed)
        return b->n_ptiles > 0 ? 1 : 0;
    const int k = staged_batch_beams_per_launch(StagedShape{b->nt, b->H, b->tb, b->dtype});
    const int n = (int)b->beams.size();
    return k > 0 ? (n + k - 1) / k : 0;
}

hs_status hs_batch_destroy(hs_batch *b)
{
    if (!b)
        return HS_OK;
    // synchronise and free on the batch's own device
    int cur = -1;
    const bool other = cudaGetDevice(&cur) == cudaSuccess && cur != b->device &&
                       cudaSetDevice(b->device) == cudaSuccess;
    cudaDeviceSynchronize();
    if (b->gexec)
        cudaGraphExecDestroy(b->gexec);
    if (b->cap_stream)
        cudaStreamDestroy(b->cap_stream);
    cudaFree(b->d_ta);
    cudaFree(b->d_order);
    cudaFree(b->d_pbeams);
    cudaFree(b->d_ptiles);
    delete b;
    if (other)
        cudaSetDevice(cur);
    return HS_OK;
}

} // extern "C"
