// hs_internal.h -- declarations shared by the host API and the kernel files.
#pragma once

#include <cstdint>
#include <vector>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/hs.h"

namespace hs {

// Upper bound on a device wait before a kernel gives up (HS_ERR_TIMEOUT).
constexpr unsigned long long kWaitLimitNs = 2000000000ull;
// Most tries of the mbarrier wait inside the staged kernel's walk (each may
// suspend up to 1 ms; the wait also stops after kWaitLimitNs).
constexpr uint32_t kBandWaitTries = 1u << 24;

struct GenericArgs {
    const void *fop;      // plane [nt][n], dtype
    const float *fop32;   // FP32 copy for rechecks, or null
    int dtype;            // hs_dtype
    int nt;               // templates (odd)
    long long n;          // bins
    long long ld;         // row pitch (elements)
    int H;                // levels
    int index;            // hs_index
    int zround;           // hs_zround
    const float *ta;      // device thresholds [H][nt]
    float delta;          // relative error bound of 16-bit storage (0 for FP32)
    float band_abs;       // absolute error bound of 16-bit storage (FP16 subnormals)
    hs_cand *rec;         // candidate records
    uint32_t *counters;   // [0] count, [1] status
    uint32_t cap;         // record capacity
    long long f_lo, f_hi; // bin range of this launch
    const float *lmin;    // host: per level the smallest threshold over all rows (H
                          // values), a prefilter bound; null = test every row exactly
};

cudaError_t launch_generic(const GenericArgs &a, cudaStream_t s);
// The harmonic-fraction map's pair-walk kernel (hs_hfrac.cu): FP32 planes,
// symmetric rounding, H = 8 or 16.
bool hfrac_pairs_available(const GenericArgs &a);
cudaError_t launch_hfrac_pairs(const GenericArgs &a, const float *lmin_host, cudaStream_t s);

// The harmonic-fraction map's staged (TMA) kernel (hs_hfrac.cu): one launch
// per level family, tiles of tb bins by K row pairs.
struct HfracStagedLaunch {
    const void *fop;       // FP32 plane [nt][ld], 16-byte aligned
    int nt;                // templates (odd)
    long long n, ld;       // bins, row pitch (elements, a multiple of 4)
    int H, tb;             // levels (8 or 16), tile bins (64 or 128)
    const float *ta;       // device thresholds [H][nt]
    const float *lmin;     // host: per level the smallest threshold over all rows
    hs_cand *rec;
    uint32_t *counters;
    uint32_t cap;
    long long f_lo, f_hi;  // bin range of this launch
    const uint32_t *order; // device tile order over the plane's tiles, or null
};
bool hfrac_staged_available(int nt, long long n, long long ld, int H, int dtype, int index,
                            int zround, int tb);
// Adds the number of kernels launched to *launches.
cudaError_t launch_hfrac_staged(const HfracStagedLaunch &L, cudaStream_t s, int *launches);

// Staged (TMA) kernel: one CTA per tile of TB bins x all templates.
constexpr int kMaxStagedH = 16;
constexpr int kMaxGroups = 8;

struct StagedShape {
    int nt, H, tb, dtype;
};

// True when a staged kernel is compiled for this (nt, H, tile bins, dtype).
bool staged_available(const StagedShape &sh);
// Dynamic shared memory bytes, box width and total bytes per tile.
int staged_smem_bytes(const StagedShape &sh);
// Box width (elements) and rows of the span read at level m (1-based).
void staged_box(const StagedShape &sh, int m, int *width, int *rows);
// Level-group ends used by the prefilter (count returned, ends in `ends`).
int staged_groups(int H, int *ends);

struct StagedLaunch {
    StagedShape sh;
    const CUtensorMap *maps;  // host copies, H descriptors (encoded for this plane)
    const CUtensorMap *split1; // level 1 in row bands (centre, outer side), or null
    const float *tmin_host;   // prefilter thresholds [groups] (min over rows)
    const float *ta;          // device thresholds [H][nt]
    const void *fop;          // the plane (device)
    const float *fop32;       // recheck copy or null
    const uint32_t *order;    // device tile order (null = linear)
    float delta;
    float band_abs;
    hs_cand *rec;
    uint32_t *counters;
    uint32_t cap;
    long long n;
    long long ld;             // row pitch of the plane and its FP32 copy (elements)
    int tile_lo, tile_hi;     // tiles [tile_lo, tile_hi) of the order
    int grid_per_sm;          // 0: one CTA per tile; k > 0: k resident CTAs per SM
    int ring_zs, ring_stages; // > 0: the pipelined kernel, consumer groups and stages
    bool assume_nonneg;       // the caller declares the plane non-negative
    int nt_rt;                // the plane's template count (0: sh.nt); a kernel family with
                              // runtime rows serves any odd count up to its compiled one
    uint2 *pend;              // 16-bit planes with an FP32 copy: device list of marked
    uint32_t *pend_count;     // row pairs for launch_recheck (null: decided in the
    uint32_t pend_cap;        // tile); pend_count[0] is zero before the launch and
                              // launch_recheck zeroes it again
};

// Decide the pending row pairs of a 16-bit plane's staged launch from its
// FP32 copy (the FP32 path's level sums, Eq. 2 order) and append the hits.
struct RecheckLaunch {
    const uint2 *pend;
    uint32_t *pend_count;    // [0] pairs listed, [1] blocks done (both zeroed at the end)
    uint32_t pend_cap;
    const float *fop32;      // [nt][ld] FP32 copy
    long long n, ld;
    int nt, H;
    const float *ta;         // device thresholds [H][nt]
    hs_cand *rec;
    uint32_t *counters;
    uint32_t cap;
};
cudaError_t launch_recheck(const RecheckLaunch &a, cudaStream_t s);

// True when the pipelined kernel is compiled for this shape, groups and stages.
bool ring_available(const StagedShape &sh, int groups, int stages);

cudaError_t launch_staged(const StagedLaunch &a, cudaStream_t s);

// Batched form: many planes (beams) of one shape.  Each launch carries the
// descriptors of up to staged_batch_beams_per_launch() beams in its
// parameter block; launch_staged_batch clears the beams' counters and issues
// as many launches as the beam count needs.
struct StagedBatchBeam {
    CUtensorMap maps[kMaxStagedH]; // host copies, H descriptors
    CUtensorMap split1[2];         // level 1 in row bands (centre, outer side)
    const float *fop32;
    long long n, ld;
    hs_cand *rec;
    uint32_t *counters;
    uint32_t cap;
    int tiles;
};

struct StagedBatch {
    StagedShape sh;
    const float *tmin_host;
    const float *ta;
    float delta, band_abs;
    const StagedBatchBeam *beams; // host array
    int n_beams;
    const uint32_t *order;        // device: tile order of each beam, concatenated (or null)
    int grid_per_sm;              // 0: one CTA per tile; k > 0: k resident CTAs per SM
    int sms;
    bool assume_nonneg;           // the caller declares every plane non-negative
};

bool staged_batch_available(const StagedShape &sh);

// Packed batch: the beams lie side by side along the bins of one plane
// [sh.nt][ld]; one set of descriptors (encode_plane_maps of the whole plane)
// and one launch (after a kernel that clears every beam's counters) cover
// them all.  Per-beam records live in device memory.
struct PackedBeam {
    long long off;       // first bin of the beam in the packed plane (16-byte multiple)
    long long n;         // bins of the beam
    hs_cand *rec;
    uint32_t *counters;  // [0] count, [1] status
    uint32_t cap;
    uint32_t pad;
};

struct PackedBatch {
    StagedShape sh;
    const CUtensorMap *maps;   // H span descriptors of the packed plane (host copies)
    const CUtensorMap *split1; // level-1 band descriptors of the packed plane
    const float *tmin_host;
    const float *ta;
    const float *fop32;        // FP32 copy of the packed plane, or null
    const uint2 *tiles;        // device: (beam, tile) per slot, in run order
    const PackedBeam *beams;   // device
    int n_beams;
    int n_tiles;
    long long ld;
    float delta, band_abs;
    int grid_per_sm;           // 0: one CTA per tile
    int sms;
    bool assume_nonneg;
};

cudaError_t launch_packed_batch(const PackedBatch &a, cudaStream_t s);
int staged_batch_beams_per_launch(const StagedShape &sh);

} // namespace hs
struct hs_batch;
namespace hs {
// Install beams whose descriptors the caller encoded already (the serving
// engine keeps one set per slot): uploads their tile order on s.
hs_status batch_set_prepared(hs_batch *b, const StagedBatchBeam *beams, int n_beams,
                             cudaStream_t s);

// Shared host helpers (hs_api.cu)
// Tile order of a plane of n_tiles tiles: 1 = linear, 2 = octave, 3 = semitone,
// 4 = 53 steps to the octave.
std::vector<uint32_t> tile_order(int n_tiles, int kind);
// The same order restricted to the tiles [tile_lo, tile_hi) (keys of their
// own tile indices).
std::vector<uint32_t> tile_order_range(int tile_lo, int tile_hi, int kind);
CUresult encode_tensor_map(CUtensorMap *map, int dtype, const void *base, long long n_bins,
                           long long ld, int n_templates, int box_w, int box_rows);
// The staged kernel's descriptors of one plane [sh.nt][n_bins] (row pitch
// ld): the H span boxes, then level 1 in row bands (centre rows
// [Z - Z/2, Z + Z/2], and Z - Z/2 rows for one outer side).
CUresult encode_plane_maps(const StagedShape &sh, const void *base, long long n_bins,
                           long long ld, CUtensorMap *maps, CUtensorMap *split1);
// Error bounds of 16-bit storage for H levels: the relative error of a
// stored value's sum (*delta) and the absolute one of FP16 subnormals
// (*band_abs); both 0 for FP32.
void storage_error(int dtype, int H, float *delta, float *band_abs);
// Prefilter bound of each level group: the smallest threshold of the group
// over all rows, lowered for 16-bit storage error and for the fast pass's
// summation order.  Returns the number of groups.
int group_bounds(const float *ta, int n_templates, int H, float delta, float band_abs,
                 float *out);
cudaError_t launch_staged_batch(const StagedBatch &a, cudaStream_t s);

} // namespace hs
