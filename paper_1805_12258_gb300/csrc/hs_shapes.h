// hs_shapes.h -- the registry of compiled staged-kernel shapes.  Each
// hs_k_*.cu file instantiates one family of shapes and returns their entry
// points; hs_staged.cu looks a shape up there.
#pragma once

#include <cuda_runtime.h>

#include "hs_internal.h"

namespace hs {

using PlaneFn = cudaError_t (*)(const StagedLaunch &, cudaStream_t);
using BatchFn = cudaError_t (*)(const StagedBatch &, cudaStream_t);
using PackedFn = cudaError_t (*)(const PackedBatch &, cudaStream_t);

// One plane shape: its stage, its boxes, the sign-checked kernel (every
// launch form) and the kernel for planes declared non-negative (or null).
struct ShapeEntry {
    StagedShape sh;
    int smem;
    void (*box)(int m, int *w, int *rows);
    PlaneFn checked;
    PlaneFn nonneg;
    bool rows_rt;   // serves every odd template count up to sh.nt (runtime rows)
};

// A shape with batched kernels: beams per launch, the descriptor-carrying
// launches and the packed-plane launch.
struct BatchEntry {
    StagedShape sh;
    int beams_per_launch;
    BatchFn batch;
    PackedFn packed;
};

// A pipelined variant of a plane shape.
struct RingEntry {
    StagedShape sh;
    int groups, stages;
    PlaneFn launch;
};

// Registration functions, one per hs_k_*.cu file: each returns the number of
// entries and points *out at a static table.
int plane_shapes_85x16_f32(const ShapeEntry **out);
int plane_shapes_85x16_f32_widths(const ShapeEntry **out);
int ring_shapes_85x16_f32(const RingEntry **out);
int batch_shapes_85x16_f32(const BatchEntry **out);
int plane_shapes_85x16_lowp(const ShapeEntry **out);
int batch_shapes_85x16_lowp(const BatchEntry **out);
int plane_shapes_21x8(const ShapeEntry **out);
int plane_shapes_rows_h16(const ShapeEntry **out);
int plane_shapes_rows_h8(const ShapeEntry **out);
int batch_shapes_21x8(const BatchEntry **out);

} // namespace hs
