// hs_hfrac.cu -- the harmonic-fraction index map on FP32 planes:
//   S_k(z, f) = sum over h = 1..k of FOP(rho(z h / k), floor(f h / k)),
// rho the symmetric rounding, every sum in ascending h, each level tested
// against its threshold (Section III's detection, on the sums of the map
// written out as "(f h/k, z h/k)").
//
// Each thread owns one bin f and walks mirrored row pairs (+zz, -zz): under
// the symmetric rounding both rows of a pair read rows +-floor(zz h/k) at the
// same bin floor(f h/k), so the pair shares every index and its two sums are
// formed with packed FP32 adds.  The levels share terms (term h/k of level k
// is term (h K/k)/K of any level K that k divides), so the levels are summed
// in families {k | K} that load level K's K terms once (100 loads per point
// for H = 16 instead of 136).  The family is the outer loop, so each family's
// K bin offsets are computed once per thread, and the row pairs the inner
// one.  A level's sum is compared with the smallest threshold of that level
// over all rows first; only a sum above it reads its rows' own thresholds.
#include <algorithm>

#include "hs_device.cuh"
#include "hs_internal.h"

namespace hs {
namespace {

constexpr bool fam_head(int K, int H)
{
    for (int M = 2 * K; M <= H; M += K)
        if (fam_head(M, H))
            return false;
    return true;
}
constexpr int fam_of(int k, int H)
{
    for (int M = H; M >= k; --M)
        if (M % k == 0 && fam_head(M, H))
            return M;
    return k;
}

template <int H>
struct LevelBounds {
    float lmin[H]; // per level: the smallest threshold over all rows (-inf: none)
};

template <int H>
__global__ void __launch_bounds__(128)
    hfrac_pair_kernel(const GenericArgs a, const LevelBounds<H> lb, int pairs_per_block)
{
    const float *plane = static_cast<const float *>(a.fop);
    const int Z = (a.nt - 1) / 2;
    const long long f64 = a.f_lo + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = f64 < a.f_hi;
    const unsigned f = (unsigned)(valid ? f64 : a.f_lo);
    const int zz_lo = (int)blockIdx.y * pairs_per_block;
    const int zz_hi = min(Z, zz_lo + pairs_per_block - 1);
    const float *pc = plane + (long long)Z * a.ld; // the centre row

    static_for<1, H + 1>([&](auto KK) {
        constexpr int K = KK;
        if constexpr (fam_head(K, H)) {
            // this family's bin offsets in the centre row, once per thread
            const float *tp[K];
            static_for<1, K + 1>([&](auto Hh) {
                constexpr int h = Hh;
                tp[h - 1] = pc + (f * (unsigned)h) / (unsigned)K;
            });
            for (int zz = zz_lo; zz <= zz_hi; ++zz) { // uniform over the CTA
                float2 t[K];
                static_for<1, K + 1>([&](auto Hh) {
                    constexpr int h = Hh;
                    const long long d = (long long)((zz * h) / K) * a.ld;
                    t[h - 1] = make_float2(__ldg(tp[h - 1] + d), __ldg(tp[h - 1] - d));
                });
                // the family's levels: hit masks over levels (top, bottom row)
                uint32_t ht = 0u, hb = 0u;
                float2 lv[K];
                static_for<1, K + 1>([&](auto Kk) {
                    constexpr int k = Kk;
                    if constexpr (K % k == 0 && fam_of(k, H) == K) {
                        constexpr int step = K / k;
                        float2 s = t[step - 1];
                        static_for<2, k + 1>([&](auto J) {
                            constexpr int j = J;
                            s = __fadd2_rn(s, t[j * step - 1]);
                        });
                        lv[k - 1] = s;
                        const float b = lb.lmin[k - 1];
                        if (s.x > b || s.y > b) { // rare: the rows' own thresholds
                            const float tt = __ldg(a.ta + (k - 1) * a.nt + (Z + zz));
                            const float tb = __ldg(a.ta + (k - 1) * a.nt + (Z - zz));
                            ht |= (s.x > tt ? 1u : 0u) << (k - 1);
                            hb |= (zz > 0 && s.y > tb ? 1u : 0u) << (k - 1);
                        }
                    }
                });
                if (!valid)
                    ht = hb = 0u;
                uint32_t slot =
                    warp_reserve(a.counters, (uint32_t)(__popc(ht) + __popc(hb)));
                if (ht | hb) {
                    static_for<1, K + 1>([&](auto Kk) {
                        constexpr int k = Kk;
                        if constexpr (K % k == 0 && fam_of(k, H) == K) {
                            if ((ht >> (k - 1)) & 1u)
                                put_record(a.rec, slot++, a.cap, f, zz, k, 0u, lv[k - 1].x);
                            if ((hb >> (k - 1)) & 1u)
                                put_record(a.rec, slot++, a.cap, f, -zz, k, 0u, lv[k - 1].y);
                        }
                    });
                }
            }
        }
    });
}

template <int H>
cudaError_t launch_h(const GenericArgs &a, const float *lmin_host, cudaStream_t s)
{
    LevelBounds<H> lb;
    for (int k = 0; k < H; ++k)
        lb.lmin[k] = lmin_host ? lmin_host[k] : -__builtin_huge_valf();
    const int threads = 128;
    const long long nbins = a.f_hi - a.f_lo;
    const long long bx = (nbins + threads - 1) / threads;
    const int pairs = (a.nt - 1) / 2 + 1;
    // enough CTAs to fill the GPU several times over: split the row pairs
    long long want = (8 * 152 * 8 + bx - 1) / bx;
    int ppb = (int)std::max(1LL, (pairs + want - 1) / want);
    ppb = std::max(ppb, std::min(pairs, 11)); // keep the family offsets worth their setup
    const int by = (pairs + ppb - 1) / ppb;
    hfrac_pair_kernel<H><<<dim3((unsigned)bx, (unsigned)by), threads, 0, s>>>(a, lb, ppb);
    return cudaGetLastError();
}

} // namespace

bool hfrac_pairs_available(const GenericArgs &a)
{
    return a.dtype == HS_F32 && a.index == HS_INDEX_HFRAC && a.zround == HS_ZROUND_SYMMETRIC &&
           (a.H == 8 || a.H == 16) && a.f_hi <= (1LL << 31) / a.H;
}

cudaError_t launch_hfrac_pairs(const GenericArgs &a, const float *lmin_host, cudaStream_t s)
{
    if (a.f_hi <= a.f_lo)
        return cudaSuccess;
    return a.H == 8 ? launch_h<8>(a, lmin_host, s) : launch_h<16>(a, lmin_host, s);
}

} // namespace hs
