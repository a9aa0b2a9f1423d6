// hs_recheck.cu -- the exact decision for a 16-bit plane's marked row pairs,
// from its FP32 copy.
//
// The staged kernel sums a 16-bit plane in FP32 and tests each level group
// against a bound lowered by the storage error, so it marks every row pair
// that may hold a hit; with an FP32 copy of the plane it appends those pairs
// (bin, pair) to a pending list instead of deciding them in the tile.  This
// kernel decides every pending pair: each row's H level sums are formed from
// the copy in the order of Eq. 2 (ascending m, FP32), exactly the numbers
// the FP32 path forms, and a level is a hit when its sum exceeds TA(k, z)
// (Section III).  The records therefore equal the FP32 path's.  One thread
// per pair loads both rows' H copy values at once, so the pairs' copy reads
// are all in flight together rather than one tile's pair after another.
#include "hs_device.cuh"
#include "hs_internal.h"

namespace hs {
namespace {

constexpr int kMaxH = 16;

#ifdef HS_CHECK_BOUNDS
constexpr bool kCheck = true;
#else
constexpr bool kCheck = false;
#endif

// pend_count[0]: pairs listed; pend_count[1]: blocks of this kernel done.
// The last block to finish zeroes both for the next run.
__global__ void __launch_bounds__(256) recheck_kernel(const RecheckLaunch a)
{
    // launched as a programmatic dependent of the summing kernel: wait until
    // that grid has completed and its writes are visible
    asm volatile("griddepcontrol.wait;" ::: "memory");
    uint32_t *pc = a.pend_count;
    const uint32_t count = min(*reinterpret_cast<volatile uint32_t *>(pc), a.pend_cap);
    const int Z = (a.nt - 1) / 2;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t stride = gridDim.x * blockDim.x;
    // whole warps iterate together (warp_reserve needs every lane)
    for (uint32_t w0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); w0 < count; w0 += stride) {
        const uint32_t i = w0 + lane;
        const bool act = i < count;
        const uint2 e = act ? a.pend[i] : make_uint2(0u, 0u);
        const uint32_t f = e.x;
        const int zz = (int)e.y;
        bool ok = act;
        if (kCheck && act && (zz > Z || (long long)f >= a.n)) {
            set_status(a.counters, HS_ERR_BOUNDS);
            ok = false;
        }
        // the rows' copy values and thresholds, all loads issued together
        float wt[kMaxH], wb[kMaxH], tt[kMaxH], tb[kMaxH];
#pragma unroll
        for (int m = 1; m <= kMaxH; ++m) {
            wt[m - 1] = wb[m - 1] = 0.f;
            tt[m - 1] = tb[m - 1] = __int_as_float(0x7f800000);
            if (ok && m <= a.H) {
                const int r = zz / m; // symmetric rounding: rows +-floor(zz/m)
                const long long b = (long long)(f / (uint32_t)m);
                wt[m - 1] = __ldg(a.fop32 + (long long)(Z + r) * a.ld + b);
                tt[m - 1] = __ldg(a.ta + (m - 1) * a.nt + (Z + zz));
                if (zz > 0) {
                    wb[m - 1] = __ldg(a.fop32 + (long long)(Z - r) * a.ld + b);
                    tb[m - 1] = __ldg(a.ta + (m - 1) * a.nt + (Z - zz));
                }
            }
        }
        uint32_t ht = 0u, hb = 0u;
        float ct = 0.f, cb = 0.f;
#pragma unroll
        for (int m = 1; m <= kMaxH; ++m) {
            if (m <= a.H) {
                ct = (m == 1) ? wt[0] : ct + wt[m - 1];
                cb = (m == 1) ? wb[0] : cb + wb[m - 1];
                wt[m - 1] = ct;
                wb[m - 1] = cb;
                ht |= (ct > tt[m - 1] ? 1u : 0u) << (m - 1);
                hb |= (cb > tb[m - 1] ? 1u : 0u) << (m - 1);
            }
        }
        uint32_t slot = warp_reserve(a.counters, (uint32_t)(__popc(ht) + __popc(hb)));
#pragma unroll
        for (int m = 1; m <= kMaxH; ++m)
            if ((ht >> (m - 1)) & 1u)
                put_record(a.rec, slot++, a.cap, f, zz, m, 0u, wt[m - 1]);
#pragma unroll
        for (int m = 1; m <= kMaxH; ++m)
            if ((hb >> (m - 1)) & 1u)
                put_record(a.rec, slot++, a.cap, f, -zz, m, 0u, wb[m - 1]);
    }
    __syncthreads(); // every thread of the block has read the count
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(pc + 1, 1u) == gridDim.x - 1) {
            pc[0] = 0u;
            pc[1] = 0u;
        }
    }
}

} // namespace

cudaError_t launch_recheck(const RecheckLaunch &a, cudaStream_t s)
{
    if (a.H < 1 || a.H > kMaxH)
        return cudaErrorInvalidValue;
    // a small grid: the pending list holds thousands of pairs on a plane
    // with signals and a few on noise; grid-stride covers any count.  A
    // programmatic dependent launch: its setup overlaps the summing kernel's
    // last tiles, its blocks start when that kernel has finished.
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(152);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, recheck_kernel, a);
}

} // namespace hs
