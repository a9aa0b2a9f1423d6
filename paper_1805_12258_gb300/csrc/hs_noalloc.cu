// hs_noalloc.cu -- harmonic summing without device allocation.
//
// hs_run_noalloc serves callers that may not allocate device memory: code
// embedded in a host framework that has reserved all device memory for its
// own pool (a stray cudaMalloc there fails or fragments the pool), and
// latency-critical loops that cannot afford cudaMalloc/cudaFree, which may
// synchronise the whole device.  It runs the same kernels as hs_run, but the
// one piece of scratch those kernels read besides their inputs and outputs,
// the threshold table, lives in a fixed array in the library's own device
// image instead of a plan allocation, and tiles run in linear order (no
// order table).
#include <cmath>
#include <string>

#include "hs_internal.h"

namespace {

// Largest threshold table (H * n_templates floats) the static array holds:
// 16384 floats = 64 KiB, e.g. 85 templates x 32 levels or 1023 x 16.
constexpr int kNoAllocMaxThresholds = 16384;

// Scratch for hs_run_noalloc, in the device image: every GPU that loads the
// library holds it until the process exits.  All calls share it.
__device__ __align__(256) float g_noalloc_ta[kNoAllocMaxThresholds];

thread_local std::string g_err;

hs_status fail(hs_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

// Device address of the static table for the current device.  It is looked
// up on every call, with the caller's device current, so a context made
// again (after cudaDeviceReset) never receives a stale address; after the
// first call on a device the lookup is a host-side table read.  The first
// call on a device may load the library's module there.
hs_status table_address(float **out)
{
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_ta);
    if (e != cudaSuccess || !ptr)
        return fail(HS_ERR_CUDA, std::string("cudaGetSymbolAddress(static thresholds): ") +
                                     cudaGetErrorString(e));
    *out = static_cast<float *>(ptr);
    return HS_OK;
}

} // namespace

extern "C" hs_status hs_run_noalloc(int n_templates, int64_t n_bins, int H,
                                    const float *thresholds, const void *fop,
                                    hs_stream_t stream, const hs_cand_buf *cands)
{
    using namespace hs;
    if (n_templates < 1 || n_templates % 2 == 0 || n_templates > 32767)
        return fail(HS_ERR_INVALID, "n_templates must be odd and in [1, 32767]");
    if (n_bins < 1 || n_bins > 0x7fffffffLL)
        return fail(HS_ERR_INVALID, "n_bins must be in [1, 2^31-1]");
    if (H < 1 || H > 32)
        return fail(HS_ERR_INVALID, "H must be in [1, 32]");
    if ((long long)H * n_templates > kNoAllocMaxThresholds)
        return fail(HS_ERR_INVALID, "H * n_templates exceeds the 16384-entry static threshold "
                                    "table of hs_run_noalloc; use a plan");
    if (!thresholds)
        return fail(HS_ERR_INVALID, "thresholds is null");
    for (long long i = 0; i < (long long)H * n_templates; ++i)
        if (!std::isfinite(thresholds[i]))
            return fail(HS_ERR_INVALID, "thresholds must be finite");
    if (!fop || reinterpret_cast<uintptr_t>(fop) % 16 != 0)
        return fail(HS_ERR_INVALID, "plane pointer must be non-null and 16-byte aligned");
    if (!cands || !cands->count || (cands->capacity > 0 && !cands->records) ||
        reinterpret_cast<uintptr_t>(cands->records) % 16 != 0)
        return fail(HS_ERR_INVALID, "candidate buffer must hold a count pointer and 16-byte "
                                    "aligned records");

    float *ta = nullptr;
    hs_status st = table_address(&ta);
    if (st != HS_OK)
        return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t ta_bytes = sizeof(float) * (size_t)H * n_templates;
    cudaError_t e = cudaMemcpyAsync(ta, thresholds, ta_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(cands->count, 0, 2 * sizeof(uint32_t), s);
    if (e != cudaSuccess)
        return fail(HS_ERR_CUDA, std::string("staging thresholds: ") + cudaGetErrorString(e));

    const int tb = 128;
    const StagedShape sh{n_templates, H, tb, HS_F32};
    if (staged_available(sh) && (n_bins * 4) % 16 == 0) {
        // prefilter bounds per level group, as a plan computes them
        float tmin[kMaxGroups];
        group_bounds(thresholds, n_templates, H, 0.f, 0.f, tmin);
        // the plan path's descriptors (host-side encoding, no allocation)
        CUtensorMap maps[kMaxStagedH];
        for (int m = 1; m <= H; ++m) {
            int w = 0, rows = 0;
            staged_box(sh, m, &w, &rows);
            if (encode_tensor_map(&maps[m - 1], HS_F32, fop, n_bins, n_bins, n_templates, w,
                                  rows) != CUDA_SUCCESS)
                return fail(HS_ERR_CUDA, "cuTensorMapEncodeTiled failed");
        }
        StagedLaunch L{};
        L.sh = sh;
        L.maps = maps;
        L.tmin_host = tmin;
        L.ta = ta;
        L.fop32 = nullptr;
        L.order = nullptr;
        L.delta = 0.f;
        L.band_abs = 0.f;
        L.rec = cands->records;
        L.counters = cands->count;
        L.cap = cands->capacity;
        L.n = n_bins;
        L.ld = n_bins;
        L.tile_lo = 0;
        L.tile_hi = (int)((n_bins + tb - 1) / tb);
        L.nt_rt = n_templates;
        e = launch_staged(L, s);
    } else {
        GenericArgs a{};
        a.fop = fop;
        a.fop32 = nullptr;
        a.dtype = HS_F32;
        a.nt = n_templates;
        a.n = n_bins;
        a.ld = n_bins;
        a.H = H;
        a.index = HS_INDEX_STRETCH;
        a.zround = HS_ZROUND_SYMMETRIC;
        a.ta = ta;
        a.delta = 0.f;
        a.band_abs = 0.f;
        a.rec = cands->records;
        a.counters = cands->count;
        a.cap = cands->capacity;
        a.f_lo = 0;
        a.f_hi = n_bins;
        e = launch_generic(a, s);
    }
    if (e != cudaSuccess)
        return fail(HS_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return HS_OK;
}

extern "C" const char *hs_noalloc_last_error(void) { return g_err.c_str(); }
