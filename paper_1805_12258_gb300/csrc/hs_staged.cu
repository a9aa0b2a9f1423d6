// hs_staged.cu -- dispatch of the staged kernel: finds a plan's, batch's or
// launch's shape among the families the hs_k_*.cu files compile (the device
// code is in hs_staged.cuh) and calls its entry point.
#include <mutex>
#include <vector>

#include "hs_shapes.h"
#include "hs_staged.cuh"

namespace hs {
namespace {

bool same(const StagedShape &a, const StagedShape &b)
{
    return a.nt == b.nt && a.H == b.H && a.tb == b.tb && a.dtype == b.dtype;
}

struct Registry {
    std::vector<ShapeEntry> planes;
    std::vector<BatchEntry> batches;
    std::vector<RingEntry> rings;
};

const Registry &registry()
{
    static Registry r;
    static std::once_flag once;
    std::call_once(once, [] {
        auto add_planes = [](int (*fn)(const ShapeEntry **)) {
            const ShapeEntry *e = nullptr;
            const int n = fn(&e);
            r.planes.insert(r.planes.end(), e, e + n);
        };
        auto add_batches = [](int (*fn)(const BatchEntry **)) {
            const BatchEntry *e = nullptr;
            const int n = fn(&e);
            r.batches.insert(r.batches.end(), e, e + n);
        };
        add_planes(plane_shapes_85x16_f32);
        add_planes(plane_shapes_85x16_f32_widths);
        add_planes(plane_shapes_85x16_lowp);
        add_planes(plane_shapes_21x8);
        add_planes(plane_shapes_rows_h16);
        add_planes(plane_shapes_rows_h8);
        add_batches(batch_shapes_85x16_f32);
        add_batches(batch_shapes_85x16_lowp);
        add_batches(batch_shapes_21x8);
        const RingEntry *e = nullptr;
        const int n = ring_shapes_85x16_f32(&e);
        r.rings.insert(r.rings.end(), e, e + n);
    });
    return r;
}

// The shape's own kernel, else the smallest family with runtime rows that
// holds its template count at the same levels, tile width and dtype.
const ShapeEntry *find_plane(const StagedShape &sh)
{
    const ShapeEntry *best = nullptr;
    for (const ShapeEntry &e : registry().planes) {
        if (!e.rows_rt && same(e.sh, sh))
            return &e;
        if (e.rows_rt && e.sh.H == sh.H && e.sh.tb == sh.tb && e.sh.dtype == sh.dtype &&
            sh.nt <= e.sh.nt && sh.nt % 2 == 1 && (!best || e.sh.nt < best->sh.nt))
            best = &e;
    }
    return best;
}

const BatchEntry *find_batch(const StagedShape &sh)
{
    for (const BatchEntry &e : registry().batches)
        if (same(e.sh, sh))
            return &e;
    return nullptr;
}

} // namespace

bool staged_available(const StagedShape &sh) { return find_plane(sh) != nullptr; }

int staged_smem_bytes(const StagedShape &sh)
{
    const ShapeEntry *e = find_plane(sh);
    return e ? e->smem : -1;
}

void staged_box(const StagedShape &sh, int m, int *width, int *rows)
{
    *width = *rows = 0;
    if (const ShapeEntry *e = find_plane(sh))
        e->box(m, width, rows);
}

int staged_batch_beams_per_launch(const StagedShape &sh)
{
    const BatchEntry *e = find_batch(sh);
    return e ? e->beams_per_launch : 0;
}

bool staged_batch_available(const StagedShape &sh) { return find_batch(sh) != nullptr; }

cudaError_t launch_staged_batch(const StagedBatch &a, cudaStream_t s)
{
    const BatchEntry *e = find_batch(a.sh);
    return e ? e->batch(a, s) : cudaErrorInvalidValue;
}

cudaError_t launch_packed_batch(const PackedBatch &a, cudaStream_t s)
{
    const BatchEntry *e = find_batch(a.sh);
    return e ? e->packed(a, s) : cudaErrorInvalidValue;
}

int staged_groups(int H, int *ends)
{
    int g = 0;
    for (int m = 1; m <= H; ++m)
        if (group_end(m, H))
            ends[g++] = m;
    return g;
}

bool ring_available(const StagedShape &sh, int groups, int stages)
{
    for (const RingEntry &e : registry().rings)
        if (same(e.sh, sh) && e.groups == groups && e.stages == stages)
            return true;
    return false;
}

cudaError_t launch_staged(const StagedLaunch &a, cudaStream_t s)
{
    if (a.ring_zs > 0) {
        for (const RingEntry &e : registry().rings)
            if (same(e.sh, a.sh) && e.groups == a.ring_zs && e.stages == a.ring_stages)
                return e.launch(a, s);
        return cudaErrorInvalidValue;
    }
    const ShapeEntry *e = find_plane(a.sh);
    if (!e)
        return cudaErrorInvalidValue;
    if (a.assume_nonneg && a.grid_per_sm == 0 && e->nonneg)
        return e->nonneg(a, s);
    return e->checked(a, s);
}

} // namespace hs
