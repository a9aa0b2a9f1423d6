// hs_internal.h -- declarations shared by the host API and the kernel files.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/hs.h"

namespace hs {

// Upper bound on a device wait before a kernel gives up (HS_ERR_TIMEOUT).
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

struct GenericArgs {
    const void *fop;      // plane [nt][n], dtype
    const float *fop32;   // FP32 copy for rechecks, or null
    int dtype;            // hs_dtype
    int nt;               // templates (odd)
    long long n;          // bins
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
};

cudaError_t launch_generic(const GenericArgs &a, cudaStream_t s);

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
    int tile_lo, tile_hi;     // tiles [tile_lo, tile_hi) of the order
};

cudaError_t launch_staged(const StagedLaunch &a, cudaStream_t s);

} // namespace hs
