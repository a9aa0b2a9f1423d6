// hs_api.cu -- host implementation of the C ABI declared in include/hs.h:
// plan creation (validation, device threshold table, prefilter thresholds,
// tile order), kernel selection, TMA descriptor encoding, the end-to-end
// host-memory call and status reporting.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "hs_internal.h"

using namespace hs;

struct hs_plan {
    int nt = 0;
    long long n = 0;
    long long ld = 0; // row pitch (elements)
    int H = 0;
    hs_options opt{};
    int device = 0;
    int kernel = HS_KERNEL_GENERIC;
    int tb = 128;
    int ring_zs = 0, ring_stages = 0; // pipelined staged kernel (0: one CTA per tile)
    int groups = 0;
    int n_tiles = 0;
    float delta = 0.f;     // relative error bound of 16-bit storage
    float band_abs = 0.f;  // absolute error bound (FP16 subnormals)
    std::vector<float> ta;   // [H][nt]
    std::vector<float> tmin; // [groups]: min over rows and the group's levels
    std::vector<float> lmin; // [H]: per level the smallest threshold over all rows
    float *d_ta = nullptr;
    uint32_t *d_order = nullptr;
    // 16-bit planes with an FP32 copy: the marked row pairs the recheck
    // kernel decides, one list per stream the plan runs on (runs on
    // different streams may overlap), allocated at the first such run
    struct Pending {
        uint2 *pairs = nullptr;
        uint32_t *count = nullptr; // [0] pairs listed, [1] recheck blocks done
    };
    std::map<cudaStream_t, Pending> pend;
    // tile order tables of partial ranges [tile_lo, tile_hi): the plan's order
    // restricted to the range, made at the first run of that range
    std::map<std::pair<int, int>, uint32_t *> range_orders;
    std::mutex mu;                 // guards the descriptor cache and streams
    const void *map_ptr = nullptr; // plane the cached descriptors encode
    CUtensorMap maps[kMaxStagedH];
    CUtensorMap split1[2]; // level 1 in row bands: centre rows, one outer side
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> chunk_events;
    bool timing = false;             // bracket kernel launches with events
    std::vector<cudaEvent_t> tev;    // event pool: (start, stop) pairs
    size_t tev_used = 0;             // events recorded since the last query
};

namespace {

// Capacity of a plan's pending list (marked row pairs of a 16-bit plane with
// an FP32 copy): 2^19 pairs, 4 MiB.  A plane that marks more has the rest
// decided inside the staged kernel.
constexpr uint32_t kPendingPairs = 1u << 19;
// Most tile-order tables of partial ranges a plan keeps at once.
constexpr size_t kMaxRangeOrders = 64;
// Most per-stream pending lists a plan keeps at once.
constexpr size_t kMaxPendingLists = 16;

thread_local std::string g_last_error;
thread_local int g_last_launches = 0;

hs_status fail(hs_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

hs_status cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                   cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? HS_ERR_OOM : HS_ERR_CUDA;
}

size_t elem_size(int dtype) { return dtype == HS_F32 ? 4 : 2; }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

} // namespace

CUresult hs::encode_tensor_map(CUtensorMap *map, int dtype, const void *base, long long n_bins,
                               long long ld, int n_templates, int box_w, int box_rows)
{
    auto fn = encode_fn();
    if (!fn)
        return CUDA_ERROR_NOT_SUPPORTED;
    const CUtensorMapDataType dt = dtype == HS_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : dtype == HS_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                      : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const size_t es = elem_size(dtype);
    cuuint64_t dims[2] = {(cuuint64_t)n_bins, (cuuint64_t)n_templates};
    cuuint64_t strides[1] = {(cuuint64_t)ld * es};
    cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, dt, 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

CUresult hs::encode_plane_maps(const StagedShape &sh, const void *base, long long n_bins,
                               long long ld, CUtensorMap *maps, CUtensorMap *split1)
{
    int w = 0, rows = 0;
    for (int m = 1; m <= sh.H; ++m) {
        staged_box(sh, m, &w, &rows);
        const CUresult r =
            encode_tensor_map(&maps[m - 1], sh.dtype, base, n_bins, ld, sh.nt, w, rows);
        if (r != CUDA_SUCCESS)
            return r;
    }
    staged_box(sh, 1, &w, &rows);
    const int z = (sh.nt - 1) / 2, rb = z / 2;
    const CUresult r =
        encode_tensor_map(&split1[0], sh.dtype, base, n_bins, ld, sh.nt, w, 2 * rb + 1);
    if (r != CUDA_SUCCESS)
        return r;
    return encode_tensor_map(&split1[1], sh.dtype, base, n_bins, ld, sh.nt, w,
                             std::max(1, z - rb));
}

void hs::storage_error(int dtype, int H, float *delta, float *band_abs)
{
    *delta = 0.f;
    *band_abs = 0.f;
    if (dtype == HS_BF16) {
        *delta = (float)((std::ldexp(1.0, -8) + H * std::ldexp(1.0, -22)) * 1.01);
    } else if (dtype == HS_F16) {
        *delta = (float)((std::ldexp(1.0, -11) + H * std::ldexp(1.0, -22)) * 1.01);
        *band_abs = (float)(H * std::ldexp(1.0, -24));
    }
}

int hs::group_bounds(const float *ta, int n_templates, int H, float delta, float band_abs,
                     float *out)
{
    int ends[kMaxGroups];
    const int groups = staged_groups(H, ends);
    double lowered[kMaxGroups], scale = 0.0;
    int a = 1;
    for (int g = 0; g < groups; ++g) {
        double t = INFINITY;
        for (int k = a; k <= ends[g]; ++k)
            for (int r = 0; r < n_templates; ++r)
                t = std::min(t, (double)ta[(size_t)(k - 1) * n_templates + r]);
        // A hit needs s (1 + delta) > t - band_abs; the fast pass sums a
        // group in tree order, within 2*gamma_H of the ascending sum, so
        // the bound is lowered by a further relative H*2^-22 (> 2 gamma_H)
        lowered[g] = (t - band_abs) / (1.0 + delta);
        lowered[g] -= std::fabs(lowered[g]) * H * std::ldexp(1.0, -22);
        scale = std::max(scale, std::fabs(lowered[g]));
        a = ends[g] + 1;
    }
    // The fast pass carries the bounds inside its sums (each group's first
    // level holds bound_{g-1} - bound_g).  Near a bound every partial sum is
    // at most about twice the largest bound in magnitude, and a pair's test
    // takes fewer than 32 roundings, so an absolute 2^-16 of the largest bound
    // (> 32 * 2^-24 * 2 * max|bound|) covers the mixing of signs; far from a
    // bound the sign of d cannot change.
    const double margin = std::ldexp(scale, -16) + std::ldexp(1.0, -126);
    for (int g = 0; g < groups; ++g) {
        const double v = lowered[g] - margin;
        float lf = (float)v;
        if ((double)lf > v)
            lf = std::nextafter(lf, -INFINITY);
        out[g] = lf;
    }
    return groups;
}

namespace hs {
// Tile order (kind 1 linear).  A tile at bin f reads the span at f/m for
// every m, which an earlier tile read in full; the orders put those tiles
// close in time so the span is still in L2.  Kind 2 (octave) sorts by the
// mantissa of the tile index, which serves m = 2, 4, 8, 16 exactly; kind 3
// (semitone) sorts by the fractional part of 12 log2(t), which also serves
// m = 3, 6, 9, 12 to within 0.02 of the period and m = 5, 10, 15 to within
// 0.14; kind 4 (the default) sorts by the fractional part of 53 log2(t),
// which serves m = 3, 6, 9, 12 to within 0.002 and m = 5, 10, 15 to within
// 0.07 (on the 85 x 2^21 plane: 745 against 762 MB read from DRAM).
std::vector<uint32_t> tile_order(int n_tiles, int kind)
{
    return tile_order_range(0, n_tiles, kind);
}

std::vector<uint32_t> tile_order_range(int tile_lo, int tile_hi, int kind)
{
    const int n_tiles = std::max(0, tile_hi - tile_lo);
    std::vector<uint32_t> o(n_tiles);
    for (int t = 0; t < n_tiles; ++t)
        o[t] = (uint32_t)(tile_lo + t);
    if (kind == 2) {
        auto key = [](uint32_t t) {
            if (t == 0)
                return std::make_pair(1.0, -1);
            int e = 31 - __builtin_clz(t);
            return std::make_pair((double)t / (double)(1u << e), e);
        };
        std::stable_sort(o.begin(), o.end(),
                         [&](uint32_t a, uint32_t b) { return key(a) < key(b); });
    } else if (kind == 3 || kind == 4) {
        // position of t within a twelfth of an octave: t, 2t, 4t, ... share
        // it exactly and 3t, 6t, 9t, 12t nearly (2^(19/12) = 2.9966); kind 4
        // divides the octave in 53 steps, in which 3t, 5t, 9t, 15t lie
        // nearer still (2^(84/53) = 2.9999, 2^(123/53) = 4.9897)
        const double steps = kind == 3 ? 12.0 : 53.0;
        auto key = [steps](uint32_t t) {
            if (t == 0)
                return -1.0;
            const double l = steps * std::log2((double)t);
            return l - std::floor(l);
        };
        std::vector<double> k(n_tiles);
        for (int t = 0; t < n_tiles; ++t)
            k[t] = key((uint32_t)(tile_lo + t));
        std::stable_sort(o.begin(), o.end(), [&](uint32_t a, uint32_t b) {
            return k[a - (uint32_t)tile_lo] < k[b - (uint32_t)tile_lo];
        });
    }
    return o;
}
} // namespace hs

namespace {

// The staged kernel's 2-D descriptors over the plane [nt][n], one per
// stretch factor m.
hs_status encode_maps(hs_plan *p, const void *fop)
{
    if (p->map_ptr == fop)
        return HS_OK;
    const StagedShape sh{p->nt, p->H, p->tb, p->opt.dtype};
    const CUresult r = encode_plane_maps(sh, fop, p->n, p->ld, p->maps, p->split1);
    if (r != CUDA_SUCCESS) {
        p->map_ptr = nullptr;
        char buf[96];
        std::snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d)", (int)r);
        return fail(HS_ERR_CUDA, buf);
    }
    p->map_ptr = fop;
    return HS_OK;
}

// A plan's tables live on the device that was current when it was made; a
// kernel launched with another device current would read them from there.
hs_status check_device(const hs_plan *p)
{
    int dev = -1;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device)
        return fail(HS_ERR_INVALID, "the plan belongs to another device: make that device "
                                    "current before running it");
    return HS_OK;
}

hs_status check_cands(const hs_cand_buf *c)
{
    if (!c || !c->count)
        return fail(HS_ERR_INVALID, "candidate buffer or its count pointer is null");
    if (c->capacity > 0 && !c->records)
        return fail(HS_ERR_INVALID, "candidate records pointer is null with capacity > 0");
    if (reinterpret_cast<uintptr_t>(c->records) % 16 != 0)
        return fail(HS_ERR_INVALID, "candidate records must be 16-byte aligned");
    return HS_OK;
}

// Launch the plan's kernel over bins [f_lo, f_hi) (tile-aligned for the
// staged kernel unless f_hi == n).  A partial range runs the plan's order
// restricted to its tiles (the harmonic-fraction map: linear).
hs_status launch_range(hs_plan *p, const void *fop, const float *fop32, cudaStream_t s,
                       const hs_cand_buf *c, long long f_lo, long long f_hi, bool full)
{
    cudaError_t e;
    cudaEvent_t ev_stop = nullptr;
    if (p->timing) {
        while (p->tev.size() < p->tev_used + 2) {
            cudaEvent_t ev;
            e = cudaEventCreate(&ev);
            if (e != cudaSuccess)
                return cuda_fail(e, "cudaEventCreate (timing)");
            p->tev.push_back(ev);
        }
        e = cudaEventRecord(p->tev[p->tev_used], s);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaEventRecord (timing)");
        ev_stop = p->tev[p->tev_used + 1];
        p->tev_used += 2;
    }
    int launches = 1;
    if (p->kernel == HS_KERNEL_STAGED && p->opt.index == HS_INDEX_HFRAC) {
        HfracStagedLaunch L{};
        L.fop = fop;
        L.nt = p->nt;
        L.n = p->n;
        L.ld = p->ld;
        L.H = p->H;
        L.tb = p->tb;
        L.ta = p->d_ta;
        L.lmin = p->lmin.data();
        L.rec = c->records;
        L.counters = c->count;
        L.cap = c->capacity;
        L.f_lo = f_lo;
        L.f_hi = f_hi;
        // the table only for a non-linear order (its default is linear)
        L.order = full && p->opt.order > 1 ? p->d_order : nullptr;
        launches = 0;
        e = launch_hfrac_staged(L, s, &launches);
        if (e != cudaSuccess)
            return cuda_fail(e, "harmonic-fraction staged kernel launch");
    } else if (p->kernel == HS_KERNEL_STAGED) {
        hs_status st = encode_maps(p, fop);
        if (st != HS_OK)
            return st;
        StagedLaunch L{};
        L.sh = StagedShape{p->nt, p->H, p->tb, p->opt.dtype};
        L.maps = p->maps;
        L.split1 = p->split1;
        L.tmin_host = p->tmin.data();
        L.fop = fop;
        L.ta = p->d_ta;
        L.fop32 = fop32;
        L.order = full ? p->d_order : nullptr;
        L.tile_lo = (int)(f_lo / p->tb);
        L.tile_hi = (int)((f_hi + p->tb - 1) / p->tb);
        if (!full && p->d_order && p->opt.order != 1) {
            // a band or chunk: the plan's order restricted to its tiles
            const auto key = std::make_pair(L.tile_lo, L.tile_hi);
            auto it = p->range_orders.find(key);
            if (it == p->range_orders.end()) {
                if (p->range_orders.size() >= kMaxRangeOrders) {
                    // many distinct ranges (a sliding window, say): start over
                    // rather than grow, once no stream of the device can still
                    // read the old tables (rare: a device-wide wait)
                    e = cudaDeviceSynchronize();
                    if (e != cudaSuccess)
                        return cuda_fail(e, "cudaDeviceSynchronize (range orders)");
                    for (auto &kv : p->range_orders)
                        cudaFree(kv.second);
                    p->range_orders.clear();
                }
                const int kind = p->opt.order != 0 ? p->opt.order : 4;
                const std::vector<uint32_t> ord = tile_order_range(L.tile_lo, L.tile_hi, kind);
                uint32_t *d = nullptr;
                e = cudaMalloc(&d, sizeof(uint32_t) * std::max<size_t>(1, ord.size()));
                if (e == cudaSuccess)
                    e = cudaMemcpy(d, ord.data(), sizeof(uint32_t) * ord.size(),
                                   cudaMemcpyHostToDevice);
                if (e != cudaSuccess) {
                    cudaFree(d);
                    return cuda_fail(e, "tile order of a range");
                }
                it = p->range_orders.emplace(key, d).first;
            }
            L.order = it->second;
            L.tile_hi -= L.tile_lo;
            L.tile_lo = 0;
        }
        L.delta = p->delta;
        L.band_abs = p->band_abs;
        L.rec = c->records;
        L.counters = c->count;
        L.cap = c->capacity;
        L.n = p->n;
        L.ld = p->ld;
        L.grid_per_sm = p->opt.grid_per_sm;
        L.ring_zs = p->ring_zs;
        L.assume_nonneg = p->opt.assume_nonneg != 0;
        L.ring_stages = p->ring_stages;
        L.nt_rt = p->nt;
        const bool defer = fop32 != nullptr && p->opt.dtype != HS_F32 && p->ring_stages == 0;
        if (defer) {
            if (p->pend.size() >= kMaxPendingLists && p->pend.find(s) == p->pend.end()) {
                // many streams (a new one per call, say): start over rather
                // than keep 4 MiB for each, once no stream can still use them
                e = cudaDeviceSynchronize();
                if (e != cudaSuccess)
                    return cuda_fail(e, "cudaDeviceSynchronize (pending lists)");
                for (auto &kv : p->pend) {
                    cudaFree(kv.second.pairs);
                    cudaFree(kv.second.count);
                }
                p->pend.clear();
            }
            hs_plan::Pending &pd = p->pend[s];
            if (!pd.pairs) {
                // the count and the recheck kernel's done-counter start at
                // zero; that kernel zeroes both again at the end of each run
                e = cudaMalloc(&pd.pairs, sizeof(uint2) * kPendingPairs);
                if (e == cudaSuccess)
                    e = cudaMalloc(&pd.count, 2 * sizeof(uint32_t));
                if (e == cudaSuccess)
                    e = cudaMemset(pd.count, 0, 2 * sizeof(uint32_t));
                if (e != cudaSuccess) {
                    cudaFree(pd.pairs);
                    cudaFree(pd.count);
                    p->pend.erase(s);
                    return cuda_fail(e, "pending list");
                }
            }
            L.pend = pd.pairs;
            L.pend_count = pd.count;
            L.pend_cap = kPendingPairs;
        }
        e = launch_staged(L, s);
        if (e == cudaSuccess && defer) {
            RecheckLaunch R{};
            R.pend = L.pend;
            R.pend_count = L.pend_count;
            R.pend_cap = kPendingPairs;
            R.fop32 = fop32;
            R.n = p->n;
            R.ld = p->ld;
            R.nt = p->nt;
            R.H = p->H;
            R.ta = p->d_ta;
            R.rec = c->records;
            R.counters = c->count;
            R.cap = c->capacity;
            e = launch_recheck(R, s);
            launches = 2;
        }
        if (e != cudaSuccess)
            return cuda_fail(e, "staged kernel launch");
    } else {
        GenericArgs a{};
        a.fop = fop;
        a.fop32 = fop32;
        a.dtype = p->opt.dtype;
        a.nt = p->nt;
        a.n = p->n;
        a.ld = p->ld;
        a.H = p->H;
        a.index = p->opt.index;
        a.zround = p->opt.zround;
        a.ta = p->d_ta;
        a.delta = p->delta;
        a.band_abs = p->band_abs;
        a.rec = c->records;
        a.counters = c->count;
        a.cap = c->capacity;
        a.f_lo = f_lo;
        a.f_hi = f_hi;
        a.lmin = p->lmin.data();
        e = launch_generic(a, s);
        if (e != cudaSuccess)
            return cuda_fail(e, "generic kernel launch");
    }
    g_last_launches += launches;
    if (ev_stop) {
        e = cudaEventRecord(ev_stop, s);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaEventRecord (timing)");
    }
    return HS_OK;
}

} // namespace

extern "C" {


hs_status hs_prefilter_bounds(const float *thresholds, int n_templates, int H, int dtype,
                              int *ends, float *bounds, int *n_groups)
{
    if (!thresholds || !ends || !bounds || !n_groups)
        return fail(HS_ERR_INVALID, "null pointer");
    if (n_templates < 1 || n_templates > 127 || n_templates % 2 == 0 || H < 2 ||
        H > kMaxStagedH || dtype < HS_F32 || dtype > HS_F16)
        return fail(HS_ERR_INVALID, "n_templates must be odd in 1..127, H in 2..16");
    float delta = 0.f, band_abs = 0.f;
    storage_error(dtype, H, &delta, &band_abs);
    const int g = staged_groups(H, ends);
    group_bounds(thresholds, n_templates, H, delta, band_abs, bounds);
    *n_groups = g;
    return HS_OK;
}

hs_status hs_tile_order(int n_tiles, int order, uint32_t *out)
{
    if (n_tiles < 0 || (n_tiles > 0 && !out) || order < 0 || order > 4)
        return fail(HS_ERR_INVALID, "n_tiles >= 0, order in 0..4 and an output array");
    const std::vector<uint32_t> o = tile_order(n_tiles, order == 0 ? 4 : order);
    std::copy(o.begin(), o.end(), out);
    return HS_OK;
}

const char *hs_status_str(hs_status s)
{
    switch (s) {
    case HS_OK: return "ok";
    case HS_ERR_INVALID: return "invalid argument";
    case HS_ERR_CUDA: return "CUDA error";
    case HS_ERR_OOM: return "out of memory";
    case HS_ERR_OVERFLOW: return "candidate buffer overflow";
    case HS_ERR_TIMEOUT: return "device wait timed out";
    case HS_ERR_UNSUPPORTED: return "unsupported";
    case HS_ERR_BUSY: return "busy (queue full or not finished)";
    case HS_ERR_BOUNDS: return "index outside its buffer (bounds-checking build)";
    }
    return "unknown status";
}

const char *hs_last_error(void) { return g_last_error.c_str(); }

int hs_last_launch_count(void) { return g_last_launches; }

hs_status hs_plan_create(hs_plan **out, int n_templates, int64_t n_bins, int H,
                         const float *thresholds, const hs_options *opt)
{
    if (!out)
        return fail(HS_ERR_INVALID, "out is null");
    *out = nullptr;
    hs_options o{};
    if (opt)
        o = *opt;
    if (n_templates < 1 || n_templates % 2 == 0 || n_templates > 32767)
        return fail(HS_ERR_INVALID, "n_templates must be odd and in [1, 32767]");
    if (n_bins < 1 || n_bins > 0x7fffffffLL)
        return fail(HS_ERR_INVALID, "n_bins must be in [1, 2^31-1]");
    if (H < 1 || H > 32)
        return fail(HS_ERR_INVALID, "H must be in [1, 32]");
    if (!thresholds)
        return fail(HS_ERR_INVALID, "thresholds is null");
    if (o.dtype < HS_F32 || o.dtype > HS_F16 || o.index < 0 || o.index > 1 || o.zround < 0 ||
        o.zround > 1 || o.kernel < 0 || o.kernel > 2 || o.order < 0 || o.order > 4 ||
        o.tile_bins < 0 || o.grid_per_sm < 0 || o.grid_per_sm > 64 || o.stages < 0 ||
        o.stages > 8 || o.z_split < 0 || o.z_split > 8 || o.assume_nonneg < 0 ||
        o.assume_nonneg > 1)
        return fail(HS_ERR_INVALID, "unknown option value");
    if (o.row_pitch != 0 && o.row_pitch < n_bins)
        return fail(HS_ERR_INVALID, "row_pitch must be 0 or at least n_bins");
    for (long long i = 0; i < (long long)H * n_templates; ++i)
        if (!std::isfinite(thresholds[i]))
            return fail(HS_ERR_INVALID, "thresholds must be finite");

    hs_plan *p = new (std::nothrow) hs_plan();
    if (!p)
        return fail(HS_ERR_OOM, "host allocation of the plan failed");
    p->nt = n_templates;
    p->n = n_bins;
    p->ld = o.row_pitch ? o.row_pitch : n_bins;
    p->H = H;
    p->opt = o;
    cudaGetDevice(&p->device);
    p->ta.assign(thresholds, thresholds + (size_t)H * n_templates);
    p->lmin.assign((size_t)H, INFINITY);
    for (int k = 0; k < H; ++k)
        for (int r = 0; r < n_templates; ++r)
            p->lmin[(size_t)k] = std::min(p->lmin[(size_t)k], p->ta[(size_t)k * n_templates + r]);
    storage_error(o.dtype, H, &p->delta, &p->band_abs);

    // kernel choice: the staged kernel needs a compiled shape, the paper's
    // index map with symmetric rounding, and 16-byte aligned rows for TMA
    const size_t es = elem_size(o.dtype);
    p->tb = o.tile_bins ? o.tile_bins : o.index == HS_INDEX_HFRAC ? 64 : 128;
    const StagedShape sh{n_templates, H, p->tb, o.dtype};
    const bool staged_ok =
        o.index == HS_INDEX_HFRAC
            ? hfrac_staged_available(n_templates, n_bins, p->ld, H, o.dtype, o.index, o.zround,
                                     p->tb)
            : staged_available(sh) && o.zround == HS_ZROUND_SYMMETRIC &&
                  (p->ld * (long long)es) % 16 == 0;
    if (o.kernel == HS_KERNEL_STAGED && !staged_ok && o.index == HS_INDEX_HFRAC) {
        delete p;
        return fail(HS_ERR_UNSUPPORTED, "no staged kernel for the harmonic-fraction map with "
                                        "these options (compiled: FP32, symmetric rounding, "
                                        "H = 8 or 16, 64 or 128 tile bins, rows a multiple "
                                        "of 16 bytes)");
    }
    if (o.kernel == HS_KERNEL_STAGED && !staged_ok) {
        delete p;
        return fail(HS_ERR_UNSUPPORTED, "no staged kernel for this shape/options "
                                        "(compiled: 85x16 and 21x8; FP32 also any odd "
                                        "template count up to 85 at H = 8 or 16 and up to "
                                        "127 at H = 16; stretch, symmetric, rows a "
                                        "multiple of 16 bytes)");
    }
    if (o.kernel == HS_KERNEL_GENERIC || !staged_ok) {
        p->kernel = HS_KERNEL_GENERIC;
        p->tb = 128;
    } else {
        p->kernel = HS_KERNEL_STAGED;
        if (o.stages > 0 && o.index == HS_INDEX_HFRAC) {
            delete p;
            return fail(HS_ERR_UNSUPPORTED, "the harmonic-fraction map has no pipelined "
                                            "staged kernel");
        }
        if (o.stages > 0) {
            const int zs = o.z_split ? o.z_split : 2;
            if (!ring_available(sh, zs, o.stages)) {
                delete p;
                return fail(HS_ERR_UNSUPPORTED, "no pipelined staged kernel for this shape, "
                                                "consumer groups and stages (compiled: 85x16 "
                                                "FP32: 128 bins with 2 or 3 groups and 3 stages, "
                                                "96 bins with 2 or 4 groups and 4 stages)");
            }
            p->ring_zs = zs;
            p->ring_stages = o.stages;
        }
    }

    cudaError_t e = cudaMalloc(&p->d_ta, sizeof(float) * p->ta.size());
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "cudaMalloc thresholds");
    }
    e = cudaMemcpy(p->d_ta, p->ta.data(), sizeof(float) * p->ta.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        hs_plan_destroy(p);
        return cuda_fail(e, "cudaMemcpy thresholds");
    }

    if (p->kernel == HS_KERNEL_STAGED) {
        p->tmin.assign((size_t)kMaxGroups, 0.f);
        p->groups = group_bounds(p->ta.data(), n_templates, H, p->delta, p->band_abs,
                                 p->tmin.data());
        p->n_tiles = (int)((n_bins + p->tb - 1) / p->tb);
        // default: 53 steps to the octave (the harmonic-fraction map: linear)
        const int kind = o.order != 0 ? o.order : o.index == HS_INDEX_HFRAC ? 1 : 4;
        std::vector<uint32_t> ord = tile_order(p->n_tiles, kind);
        e = cudaMalloc(&p->d_order, sizeof(uint32_t) * ord.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(p->d_order, ord.data(), sizeof(uint32_t) * ord.size(),
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            hs_plan_destroy(p);
            return cuda_fail(e, "tile order table");
        }
    }
    *out = p;
    return HS_OK;
}

int hs_plan_kernel(const hs_plan *p) { return p ? p->kernel : 0; }

int hs_plan_tile_bins(const hs_plan *p) { return p ? p->tb : 0; }

hs_status hs_run_checked(hs_plan *p, const void *fop, const float *fop32, hs_stream_t stream,
                         const hs_cand_buf *cands)
{
    g_last_launches = 0;
    if (!p)
        return fail(HS_ERR_INVALID, "plan is null");
    if (hs_status d = check_device(p); d != HS_OK)
        return d;
    if (!fop || reinterpret_cast<uintptr_t>(fop) % 16 != 0)
        return fail(HS_ERR_INVALID, "plane pointer must be non-null and 16-byte aligned");
    if (fop32 && p->opt.dtype == HS_F32)
        return fail(HS_ERR_INVALID, "an FP32 plan takes no recheck copy");
    if (fop32 && reinterpret_cast<uintptr_t>(fop32) % 16 != 0)
        return fail(HS_ERR_INVALID, "recheck copy must be 16-byte aligned");
    hs_status st = check_cands(cands);
    if (st != HS_OK)
        return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(cands->count, 0, 2 * sizeof(uint32_t), s);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync counters");
    std::lock_guard<std::mutex> lk(p->mu);
    return launch_range(p, fop, fop32, s, cands, 0, p->n, true);
}

hs_status hs_run(hs_plan *p, const void *fop, hs_stream_t stream, const hs_cand_buf *cands)
{
    return hs_run_checked(p, fop, nullptr, stream, cands);
}

hs_status hs_run_range(hs_plan *p, const void *fop, const float *fop32, int64_t f_lo,
                       int64_t f_hi, hs_stream_t stream, const hs_cand_buf *cands, int append)
{
    g_last_launches = 0;
    if (!p)
        return fail(HS_ERR_INVALID, "plan is null");
    if (hs_status d = check_device(p); d != HS_OK)
        return d;
    if (!fop || reinterpret_cast<uintptr_t>(fop) % 16 != 0)
        return fail(HS_ERR_INVALID, "plane pointer must be non-null and 16-byte aligned");
    if (fop32 && (p->opt.dtype == HS_F32 || reinterpret_cast<uintptr_t>(fop32) % 16 != 0))
        return fail(HS_ERR_INVALID, "bad recheck copy (FP32 plans take none; 16-byte aligned)");
    const long long unit = p->kernel == HS_KERNEL_STAGED ? p->tb : 1;
    if (f_lo < 0 || f_hi > p->n || f_lo >= f_hi || f_lo % unit != 0 ||
        (f_hi != p->n && f_hi % unit != 0))
        return fail(HS_ERR_INVALID, "need 0 <= f_lo < f_hi <= n_bins with f_lo (and f_hi "
                                    "unless it is n_bins) a multiple of hs_plan_tile_bins()");
    hs_status st = check_cands(cands);
    if (st != HS_OK)
        return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!append) {
        cudaError_t e = cudaMemsetAsync(cands->count, 0, 2 * sizeof(uint32_t), s);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaMemsetAsync counters");
    }
    std::lock_guard<std::mutex> lk(p->mu);
    return launch_range(p, fop, fop32, s, cands, f_lo, f_hi, false);
}

hs_status hs_cand_sync(const hs_cand_buf *cands, hs_stream_t stream, uint32_t *n_out)
{
    hs_status st = check_cands(cands);
    if (st != HS_OK)
        return st;
    uint32_t h[2] = {0, 0};
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(h, cands->count, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return cuda_fail(e, "reading candidate count");
    if (n_out)
        *n_out = h[0];
    if (h[1] != 0)
        return fail((hs_status)h[1], "device reported a failed bounded wait");
    if (h[0] > cands->capacity)
        return fail(HS_ERR_OVERFLOW, "more candidates than the buffer capacity");
    return HS_OK;
}

hs_status hs_run_host(hs_plan *p, const void *fop_host, void *fop_dev, const hs_cand_buf *cands,
                      hs_cand *host_records, uint32_t host_capacity, hs_stream_t stream,
                      uint32_t *n_out)
{
    return hs_run_host_checked(p, fop_host, fop_dev, nullptr, cands, host_records, host_capacity,
                               stream, n_out);
}

hs_status hs_run_host_checked(hs_plan *p, const void *fop_host, void *fop_dev,
                              const float *fop32_host, const hs_cand_buf *cands,
                              hs_cand *host_records, uint32_t host_capacity, hs_stream_t stream,
                              uint32_t *n_out)
{
    g_last_launches = 0;
    if (!p || !fop_host || !fop_dev)
        return fail(HS_ERR_INVALID, "plan, host plane and device plane must be non-null");
    if (hs_status d = check_device(p); d != HS_OK)
        return d;
    const float *fop32_dev = nullptr;
    if (fop32_host) {
        if (p->opt.dtype == HS_F32)
            return fail(HS_ERR_INVALID, "an FP32 plan takes no recheck copy");
        // rechecks read the few near-threshold points straight from the
        // page-locked host copy (mapped into the device's address space)
        void *dp = nullptr;
        if (cudaHostGetDevicePointer(&dp, const_cast<float *>(fop32_host), 0) != cudaSuccess ||
            reinterpret_cast<uintptr_t>(dp) % 16 != 0) {
            cudaGetLastError();
            return fail(HS_ERR_INVALID, "the FP32 recheck copy must be host memory the device "
                                        "can address (page-locked), 16-byte aligned");
        }
        fop32_dev = static_cast<const float *>(dp);
    }
    if (reinterpret_cast<uintptr_t>(fop_dev) % 16 != 0)
        return fail(HS_ERR_INVALID, "device plane must be 16-byte aligned");
    if (host_capacity > 0 && !host_records)
        return fail(HS_ERR_INVALID, "host_records is null with host_capacity > 0");
    hs_status st = check_cands(cands);
    if (st != HS_OK)
        return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t es = elem_size(p->opt.dtype);
    const int n_chunks = 8;
    {
        std::lock_guard<std::mutex> lk(p->mu);
        cudaError_t e = cudaSuccess;
        if (!p->copy_stream)
            e = cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking);
        while (e == cudaSuccess && (int)p->chunk_events.size() < n_chunks + 1) {
            cudaEvent_t ev;
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess)
                p->chunk_events.push_back(ev);
        }
        if (e != cudaSuccess)
            return cuda_fail(e, "creating copy stream/events");
        // the copy stream starts after work already queued on `stream`
        e = cudaEventRecord(p->chunk_events[n_chunks], s);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(p->copy_stream, p->chunk_events[n_chunks], 0);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(cands->count, 0, 2 * sizeof(uint32_t), s);
        if (e != cudaSuccess)
            return cuda_fail(e, "ordering the copy stream");
        // chunk edges: tile-aligned so each chunk's outputs need only bins
        // already copied (every source bin floor(f/m) <= f)
        const long long unit = p->kernel == HS_KERNEL_STAGED ? p->tb : 128;
        const long long units = (p->n + unit - 1) / unit;
        long long prev = 0;
        for (int c = 0; c < n_chunks; ++c) {
            long long hi = (c == n_chunks - 1) ? p->n : std::min(p->n, units * (c + 1) / n_chunks * unit);
            if (hi <= prev)
                continue;
            const size_t off = (size_t)prev * es, width = (size_t)(hi - prev) * es,
                         pitch = (size_t)p->ld * es;
            e = cudaMemcpy2DAsync(static_cast<char *>(fop_dev) + off, pitch,
                                  static_cast<const char *>(fop_host) + off, pitch, width,
                                  (size_t)p->nt, cudaMemcpyHostToDevice, p->copy_stream);
            if (e == cudaSuccess)
                e = cudaEventRecord(p->chunk_events[c], p->copy_stream);
            if (e == cudaSuccess)
                e = cudaStreamWaitEvent(s, p->chunk_events[c], 0);
            if (e != cudaSuccess)
                return cuda_fail(e, "host-to-device chunk copy");
            st = launch_range(p, fop_dev, fop32_dev, s, cands, prev, hi, false);
            if (st != HS_OK)
                return st;
            prev = hi;
        }
    }
    uint32_t n = 0;
    hs_status sync = hs_cand_sync(cands, stream, &n);
    if (sync != HS_OK && sync != HS_ERR_OVERFLOW)
        return sync;
    if (n_out)
        *n_out = n;
    const uint32_t ncopy = std::min(std::min(n, cands->capacity), host_capacity);
    if (ncopy > 0) {
        cudaError_t e = cudaMemcpyAsync(host_records, cands->records, sizeof(hs_cand) * ncopy,
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            return cuda_fail(e, "device-to-host candidate copy");
    }
    if (sync == HS_OK && n > host_capacity)
        return fail(HS_ERR_OVERFLOW, "more candidates than the host buffer capacity");
    return sync;
}

hs_status hs_plan_set_timing(hs_plan *p, int enable)
{
    if (!p)
        return fail(HS_ERR_INVALID, "plan is null");
    std::lock_guard<std::mutex> lk(p->mu);
    p->timing = enable != 0;
    return HS_OK;
}

hs_status hs_plan_kernel_time(hs_plan *p, double *total_ms, int *launches)
{
    if (!p)
        return fail(HS_ERR_INVALID, "plan is null");
    std::lock_guard<std::mutex> lk(p->mu);
    double total = 0.0;
    for (size_t i = 0; i + 1 < p->tev_used; i += 2) {
        cudaError_t e = cudaEventSynchronize(p->tev[i + 1]);
        float ms = 0.f;
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, p->tev[i], p->tev[i + 1]);
        if (e != cudaSuccess)
            return cuda_fail(e, "reading kernel timing events");
        total += ms;
    }
    if (total_ms)
        *total_ms = total;
    if (launches)
        *launches = (int)(p->tev_used / 2);
    p->tev_used = 0;
    return HS_OK;
}

hs_status hs_plan_destroy(hs_plan *p)
{
    if (!p)
        return HS_OK;
    // synchronise and free on the plan's own device
    int cur = -1;
    const bool other = cudaGetDevice(&cur) == cudaSuccess && cur != p->device &&
                       cudaSetDevice(p->device) == cudaSuccess;
    cudaDeviceSynchronize();
    cudaFree(p->d_ta);
    cudaFree(p->d_order);
    for (auto &kv : p->pend) {
        cudaFree(kv.second.pairs);
        cudaFree(kv.second.count);
    }
    for (auto &kv : p->range_orders)
        cudaFree(kv.second);
    for (cudaEvent_t ev : p->tev)
        cudaEventDestroy(ev);
    for (cudaEvent_t ev : p->chunk_events)
        cudaEventDestroy(ev);
    if (p->copy_stream)
        cudaStreamDestroy(p->copy_stream);
    delete p;
    if (other)
        cudaSetDevice(cur);
    return HS_OK;
}

hs_status hs_pack_paper(const hs_cand *c, int n_templates, uint32_t *cl1, float *cl2)
{
    if (!c || !cl1 || !cl2 || n_templates < 1 || n_templates % 2 == 0)
        return fail(HS_ERR_INVALID, "null argument or even template count");
    const int Z = (n_templates - 1) / 2;
    const int r = c->z + Z;
    if (r < 0 || r >= 128 || c->k < 1 || c->k > 8 || c->bin >= (1u << 21))
        return fail(HS_ERR_INVALID, "field does not fit the 7+3+21-bit packing");
    *cl1 = ((uint32_t)r << 24) | ((uint32_t)(c->k - 1) << 21) | c->bin;
    *cl2 = c->power;
    return HS_OK;
}

} // extern "C"
