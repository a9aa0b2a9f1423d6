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

// Level k of point (z, f) from the FP32 copy, out of line: the rechecks of
// 16-bit planes are rare and stay off the fixed kernel's registers.
__device__ __noinline__ float recheck_level(const float *fop32, int Z, long long ld, int index,
                                            int zround, int z, unsigned f, int k)
{
    float a;
    return level_value(fop32, Z, ld, index, zround, z, (long long)f, k, &a);
}

// The same computation for a level count fixed at compile time: every row
// scale z h / k and bin scale f h / k becomes a division by a constant (a
// multiply-high) instead of a runtime integer division, and the level values
// stay in registers for the record pass.  Bins are 32-bit: the launcher uses
// it when f h fits (f < 2^31 / H).
template <int NUM, int DEN, int ZR>
__device__ __forceinline__ int scale_row_c(int z)
{
    const int p = z * NUM;
    if (ZR == HS_ZROUND_FLOOR) {
        int q = p / DEN;
        if ((p % DEN) != 0 && p < 0)
            q -= 1;
        return q;
    }
    return p >= 0 ? p / DEN : -((-p) / DEN);
}

// Families of harmonic-fraction levels: K heads a family unless a multiple
// of K up to H does; level k belongs to the largest head it divides.
constexpr bool family_head(int K, int H)
{
    for (int M = 2 * K; M <= H; M += K)
        if (family_head(M, H))
            return false;
    return true;
}
constexpr int family_of(int k, int H)
{
    for (int M = H; M >= k; --M)
        if (M % k == 0 && family_head(M, H))
            return M;
    return k;
}

template <typename T, int H, int INDEX, int ZR>
__global__ void __launch_bounds__(128, 4)
    generic_fixed_kernel(GenericArgs a, int rows_per_block)
{
    const T *fop = static_cast<const T *>(a.fop);
    const int Z = (a.nt - 1) / 2;
    const long long f64 = a.f_lo + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = f64 < a.f_hi;
    const unsigned f = (unsigned)(valid ? f64 : a.f_lo);
    const int z_lo = -Z + (int)blockIdx.y * rows_per_block;
    const int z_hi = min(Z, z_lo + rows_per_block - 1);
    auto ld = [&](int row, unsigned bin) {
        return to_f32(__ldg(fop + (long long)row * a.ld + bin));
    };

    for (int z = z_lo; z <= z_hi; ++z) { // uniform over the block
        const int row = z + Z;
        float lv[H], la[H];
        if constexpr (INDEX == HS_INDEX_STRETCH) {
            float s = 0.f, ab = 0.f;
            static_for<1, H + 1>([&](auto M) {
                constexpr int m = M;
                const float v = ld(scale_row_c<1, m, ZR>(z) + Z, f / (unsigned)m);
                s = (m == 1) ? v : s + v;
                ab += fabsf(v);
                lv[m - 1] = s;
                la[m - 1] = ab;
            });
        } else {
            // levels share terms: the term h/k of level k is the term
            // (h K/k)/K of every level K that k divides, so each family
            // {k | K} loads level K's K terms once and sums its members from
            // them (100 loads per point for H = 16 instead of 136), every sum
            // in ascending h as before
            static_for<1, H + 1>([&](auto KK) {
                constexpr int K = KK;
                if constexpr (family_head(K, H)) {
                    float t[K];
                    static_for<1, K + 1>([&](auto Hh) {
                        constexpr int h = Hh;
                        t[h - 1] = ld(scale_row_c<h, K, ZR>(z) + Z,
                                      (f * (unsigned)h) / (unsigned)K);
                    });
                    static_for<1, K + 1>([&](auto Kk) {
                        constexpr int k = Kk;
                        if constexpr (K % k == 0 && family_of(k, H) == K) {
                            constexpr int step = K / k;
                            float s = 0.f, ab = 0.f;
                            static_for<1, k + 1>([&](auto J) {
                                constexpr int j = J;
                                const float v = t[j * step - 1];
                                s = (j == 1) ? v : s + v;
                                ab += fabsf(v);
                            });
                            lv[k - 1] = s;
                            la[k - 1] = ab;
                        }
                    });
                }
            });
        }
        // pass 1: hit mask over the levels; 16-bit planes re-add a possible
        // hit from the FP32 copy (rare, out of line)
        uint32_t hits = 0u;
        static_for<0, H>([&](auto Kk) {
            constexpr int k = Kk + 1;
            const float thr = __ldg(a.ta + (k - 1) * a.nt + row);
            bool hit;
            if (a.delta == 0.f || a.fop32 == nullptr) {
                hit = lv[Kk] > thr;
            } else {
                const float band = a.delta * la[Kk] + a.band_abs;
                hit = !(lv[Kk] == lv[Kk] && lv[Kk] + band < thr) &&
                      recheck_level(a.fop32, Z, a.ld, a.index, a.zround, z, f, k) > thr;
            }
            if (hit)
                hits |= 1u << Kk;
        });
        if (!valid)
            hits = 0u;
        uint32_t slot = warp_reserve(a.counters, (uint32_t)__popc(hits));
        // pass 2: the records of the hit levels
        static_for<0, H>([&](auto Kk) {
            constexpr int k = Kk + 1;
            if (hits & (1u << Kk)) {
                float power = lv[Kk];
                uint32_t flags = 0u;
                if (a.delta != 0.f) {
                    if (a.fop32 != nullptr) {
                        power = recheck_level(a.fop32, Z, a.ld, a.index, a.zround, z, f, k);
                    } else {
                        const float thr = __ldg(a.ta + (k - 1) * a.nt + row);
                        flags = HS_FLAG_LOWP | (fabsf(lv[Kk] - thr) <= a.delta * la[Kk] + a.band_abs
                                                    ? HS_FLAG_NEAR
                                                    : 0u);
                    }
                }
                put_record(a.rec, slot++, a.cap, f, z, k, flags, power);
            }
        });
    }
}

template <typename T, int H>
void launch_fixed(const GenericArgs &a, dim3 grid, int threads, int rows, cudaStream_t s)
{
    if (a.index == HS_INDEX_STRETCH) {
        if (a.zround == HS_ZROUND_FLOOR)
            generic_fixed_kernel<T, H, HS_INDEX_STRETCH, HS_ZROUND_FLOOR><<<grid, threads, 0, s>>>(a, rows);
        else
            generic_fixed_kernel<T, H, HS_INDEX_STRETCH, HS_ZROUND_SYMMETRIC><<<grid, threads, 0, s>>>(a, rows);
    } else {
        if (a.zround == HS_ZROUND_FLOOR)
            generic_fixed_kernel<T, H, HS_INDEX_HFRAC, HS_ZROUND_FLOOR><<<grid, threads, 0, s>>>(a, rows);
        else
            generic_fixed_kernel<T, H, HS_INDEX_HFRAC, HS_ZROUND_SYMMETRIC><<<grid, threads, 0, s>>>(a, rows);
    }
}

} // namespace

cudaError_t launch_generic(const GenericArgs &a, cudaStream_t s)
{
    if (a.f_hi <= a.f_lo)
        return cudaSuccess;
    if (hfrac_pairs_available(a))
        return launch_hfrac_pairs(a, a.lmin, s);
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
    // compiled level counts with 32-bit bin products take the fixed kernel
    if ((a.H == 8 || a.H == 16) && a.f_hi <= (1LL << 31) / a.H) {
        switch (a.dtype) {
        case HS_F32:
            a.H == 8 ? launch_fixed<float, 8>(a, grid, threads, rows_per_block, s)
                     : launch_fixed<float, 16>(a, grid, threads, rows_per_block, s);
            break;
        case HS_BF16:
            a.H == 8 ? launch_fixed<__nv_bfloat16, 8>(a, grid, threads, rows_per_block, s)
                     : launch_fixed<__nv_bfloat16, 16>(a, grid, threads, rows_per_block, s);
            break;
        case HS_F16:
            a.H == 8 ? launch_fixed<__half, 8>(a, grid, threads, rows_per_block, s)
                     : launch_fixed<__half, 16>(a, grid, threads, rows_per_block, s);
            break;
        default:
            return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
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
