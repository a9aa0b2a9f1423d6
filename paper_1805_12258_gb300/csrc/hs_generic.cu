// hs_generic.cu -- the shape-agnostic harmonic-summing kernel.
//
// Any odd template count, 1 <= H <= 32, both index maps (Eq. 1-2 stretch sums
// and the harmonic-fraction sums), both row roundings, FP32/BF16/FP16 planes
// and any alignment.  Each thread owns one bin f and walks a block of template
// rows; for every row it forms the H level values in registers in the order
// of Algorithm 2 (levels innermost), reading the plane through the read-only
// cache, tests each against TA(k, row) and appends hits with one atomic per
// warp.  The staged kernel (hs_staged.cu) is the fast path for the common
// shapes; this kernel is the fallback and a second implementation to check it.
#include "hs_device.cuh"
#include "hs_internal.h"

namespace hs {
namespace {

// Row read for output row z when the plane is scaled by num/den.
__device__ __forceinline__ int scale_row(int z, int num, int den, int zround)
{
    const int p = z * num;
    if (zround == HS_ZROUND_FLOOR) {
        int q = p / den;
        if ((p % den) != 0 && p < 0)
            q -= 1;
        return q;
    }
    return p >= 0 ? p / den : -((-p) / den);
}

template <typename T>
__device__ __forceinline__ float ld_plane(const T *fop, long long ld, int row, long long bin)
{
    return to_f32(__ldg(fop + (long long)row * ld + bin));
}

// Level value k (1-based) of point (z, f) of a plane with row pitch ld, and
// the sum of absolute values of its terms.  STRETCH: the cumulative Eq. 2 chain up to k, ascending m;
// HFRAC: the k terms (z*h/k, f*h/k), ascending h.
template <typename T>
__device__ float level_value(const T *fop, int Z, long long ld, int index, int zround, int z,
                            long long f, int k, float *abs_sum)
{
    float s = 0.f, a = 0.f;
    if (index == HS_INDEX_STRETCH) {
        for (int m = 1; m <= k; ++m) {
            const float v = ld_plane(fop, ld, scale_row(z, 1, m, zround) + Z, f / m);
            s = (m == 1) ? v : s + v;
            a += fabsf(v);
        }
    } else {
        for (int h = 1; h <= k; ++h) {
            const float v =
                ld_plane(fop, ld, scale_row(z, h, k, zround) + Z, (f * h) / k);
            s = (h == 1) ? v : s + v;
            a += fabsf(v);
        }
    }
    *abs_sum = a;
    return s;
}

// Decide level k of point (z, f).  Returns true on a hit with *power and
// *flags set.  For 16-bit planes (delta > 0) a possible hit is re-evaluated
// from the FP32 copy when one is given.
template <typename T>
__device__ bool decide(const T *fop, const float *fop32, int Z, long long ld, int index,
                       int zround, int z, long long f, int k, float s, float a, float thr,
                       float delta, float band_abs, float *power, uint32_t *flags)
{
    if (delta == 0.f) {
        *power = s;
        *flags = 0u;
        return s > thr;
    }
    const float band = delta * a + band_abs;
    if (fop32 != nullptr) {
        if (s == s && s + band < thr) // cannot exceed thr in FP32 (NaN is rechecked)
            return false;
        float a32;
        const float s32 = level_value(fop32, Z, ld, index, zround, z, f, k, &a32);
        *power = s32;
        *flags = 0u;
        return s32 > thr;
    }
    *power = s;
    *flags = HS_FLAG_LOWP | (fabsf(s - thr) <= band ? HS_FLAG_NEAR : 0u);
    return s > thr;
}

template <typename T>
__global__ void __launch_bounds__(128)
    generic_kernel(GenericArgs a, int rows_per_block)
{
    const T *fop = static_cast<const T *>(a.fop);
    const int Z = (a.nt - 1) / 2;
    const long long f = a.f_lo + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = f < a.f_hi;
    const long long fc = valid ? f : a.f_lo;
    const int z_lo = -Z + (int)blockIdx.y * rows_per_block;
    const int z_hi = min(Z, z_lo + rows_per_block - 1);

    for (int z = z_lo; z <= z_hi; ++z) { // uniform over the block
        const int row = z + Z;
        // pass 1: levels of this point, hit mask over k
        uint32_t hits = 0u;
        if (a.index == HS_INDEX_STRETCH) {
            float s = 0.f, ab = 0.f;
            for (int m = 1; m <= a.H; ++m) {
                const float v =
                    ld_plane(fop, a.ld, scale_row(z, 1, m, a.zround) + Z, fc / m);
                s = (m == 1) ? v : s + v;
                ab += fabsf(v);
                float pw;
                uint32_t fl;
                if (decide(fop, a.fop32, Z, a.ld, a.index, a.zround, z, fc, m, s, ab,
                           __ldg(a.ta + (m - 1) * a.nt + row), a.delta, a.band_abs, &pw, &fl))
                    hits |= 1u << (m - 1);
            }
        } else {
            for (int k = 1; k <= a.H; ++k) {
                float ab;
                const float s = level_value(fop, Z, a.ld, a.index, a.zround, z, fc, k, &ab);
                float pw;
                uint32_t fl;
                if (decide(fop, a.fop32, Z, a.ld, a.index, a.zround, z, fc, k, s, ab,
                           __ldg(a.ta + (k - 1) * a.nt + row), a.delta, a.band_abs, &pw, &fl))
                    hits |= 1u << (k - 1);
            }
        }
        if (!valid)
            hits = 0u;
        // one atomic per warp for the warp's hits of this row
        uint32_t slot = warp_reserve(a.counters, (uint32_t)__popc(hits));
        // pass 2 (rare): recompute the hit levels and write their records
        while (hits) {
            const int k = __ffs(hits);
            hits &= hits - 1u;
            float ab;
            const float s = level_value(fop, Z, a.ld, a.index, a.zround, z, fc, k, &ab);
            float pw;
            uint32_t fl;
            decide(fop, a.fop32, Z, a.ld, a.index, a.zround, z, fc, k, s, ab,
                   __ldg(a.ta + (k - 1) * a.nt + row), a.delta, a.band_abs, &pw, &fl);
            put_record(a.rec, slot++, a.cap, (uint32_t)fc, z, k, fl, pw);
        }
    }
}

} // namespace

cudaError_t launch_generic(const GenericArgs &a, cudaStream_t s)
{
    if (a.f_hi <= a.f_lo)
        return cudaSuccess;
    const int threads = 128;
    const long long nbins = a.f_hi - a.f_lo;
    const long long bx = (nbins + threads - 1) / threads;
    // enough CTAs to fill the GPU: split rows when there are few bin blocks
    int rows_per_block = a.nt;
    if (bx < 4096) {
        const long long want = (4096 + bx - 1) / bx;
        rows_per_block = (int)((a.nt + want - 1) / want);
        if (rows_per_block < 1)
            rows_per_block = 1;
    }
    const int by = (a.nt + rows_per_block - 1) / rows_per_block;
    dim3 grid((unsigned)bx, (unsigned)by);
    switch (a.dtype) {
    case HS_F32:
        generic_kernel<float><<<grid, threads, 0, s>>>(a, rows_per_block);
        break;
    case HS_BF16:
        generic_kernel<__nv_bfloat16><<<grid, threads, 0, s>>>(a, rows_per_block);
        break;
    case HS_F16:
        generic_kernel<__half><<<grid, threads, 0, s>>>(a, rows_per_block);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

} // namespace hs
