// hs_hfrac.cu -- the harmonic-fraction index map on FP32 planes:
//   S_k(z, f) = sum over h = 1..k of FOP(rho(z h / k), floor(f h / k)),
// rho the symmetric rounding, every sum in ascending h, each level tested
// against its threshold (Section III's detection, on the sums of the map
// written out as "(f h/k, z h/k)").
//
// Both kernels here give each thread one bin f and walk mirrored row pairs
// (+zz, -zz): under the symmetric rounding both rows of a pair read rows
// +-floor(zz h/k) at the same bin floor(f h/k), so the pair shares every index
// and its two sums are formed with packed FP32 adds.  The levels share terms
// (term h/k of level k is term (h K/k)/K of any level K that k divides), so
// the levels are summed in families {k | K} that load level K's K terms once
// (100 loads per point for H = 16 instead of 136).  One CTA runs one family.
// A level's sum is compared with the smallest threshold of that level over
// all rows first; only a sum above it reads its rows' own thresholds.
//
// Staged kernel (one launch per family K): a CTA takes TB bins and the K row
// pairs zz = jK .. jK + K - 1.  Because the block starts at a multiple of K,
// term h reads rows +-(jh + floor(i h/K)) for i = zz - jK: exactly h rows on
// each side.  Each term's rows arrive as two 2-D TMA boxes (top and bottom)
// of h rows and the term's bin span; a thread reads a term at its column
// register plus the step's row offset.
//
// Gather kernel (any row pitch): the same walk reading global memory through
// the read-only path, the family the grid's slowest index, the warp-uniform
// row offsets floor(zz h/K) * ld kept in a shared table.
#include <algorithm>
#include <cstring>
#include <vector>

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
constexpr int n_heads(int H)
{
    int n = 0;
    for (int K = 1; K <= H; ++K)
        n += fam_head(K, H) ? 1 : 0;
    return n;
}
// Family heads in descending order: index 0 is H (the most terms).
constexpr int head_at(int i, int H)
{
    for (int K = H, n = 0; K >= 1; --K)
        if (fam_head(K, H)) {
            if (n == i)
                return K;
            ++n;
        }
    return 0;
}
constexpr int round_up(int x, int a) { return (x + a - 1) / a * a; }

// Opt-in bounds checks (-DHS_CHECK_BOUNDS): the staged kernel tests every
// shared-memory read against its own term's box and the gather kernel every
// plane read against the plane, each threshold read against the table; an
// index outside sets HS_ERR_BOUNDS in the status word and the read is skipped
// (0 for a value, +inf for a threshold).  Never a trap.
#ifdef HS_CHECK_BOUNDS
constexpr bool kCheck = true;
#else
constexpr bool kCheck = false;
#endif

// Host counterpart of static_for: f(std::integral_constant<int, i>) for
// i = B .. E-1.
template <int B, int E, typename F>
void static_for_host(F &&f)
{
    if constexpr (E > B) {
        f(std::integral_constant<int, B>{});
        static_for_host<B + 1, E>(static_cast<F &&>(f));
    }
}

template <int H>
struct LevelBounds {
    float lmin[H]; // per level: the smallest threshold over all rows (-inf: none)
};

struct HitSink {
    const float *ta; // device thresholds [H][nt]
    hs_cand *rec;
    uint32_t *counters;
    uint32_t cap;
    int nt;
};

// The levels of family K at pair zz from its terms t[h - 1] (x: row +zz,
// y: row -zz): each level summed in ascending h and compared with the
// smallest threshold of the level over all rows; a warp any of whose lanes
// passes one takes the exact per-row tests and records the hits.
template <int H, int K>
__device__ __forceinline__ void family_levels(const float2 (&t)[K], int zz, unsigned f,
                                              bool valid, const LevelBounds<H> &lb,
                                              const HitSink &o)
{
    float2 lv[K];
    bool over = false;
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
            over = over | (s.x > b) | (s.y > b);
        }
    });
    over = over && valid;
    if (!__any_sync(0xffffffffu, over)) // the common case
        return;
    const int Z = (o.nt - 1) / 2;
    uint32_t ht = 0u, hb = 0u;
    if (over) {
        static_for<1, K + 1>([&](auto Kk) {
            constexpr int k = Kk;
            if constexpr (K % k == 0 && fam_of(k, H) == K) {
                const float2 s = lv[k - 1];
                float tt, tb;
                if (kCheck && (zz < 0 || zz > Z)) {
                    set_status(o.counters, HS_ERR_BOUNDS);
                    tt = tb = __int_as_float(0x7f800000);
                } else {
                    tt = __ldg(o.ta + (k - 1) * o.nt + (Z + zz));
                    tb = __ldg(o.ta + (k - 1) * o.nt + (Z - zz));
                }
                ht |= (s.x > tt ? 1u : 0u) << (k - 1);
                hb |= (zz > 0 && s.y > tb ? 1u : 0u) << (k - 1);
            }
        });
    }
    uint32_t slot = warp_reserve(o.counters, (uint32_t)(__popc(ht) + __popc(hb)));
    if (ht | hb) {
        static_for<1, K + 1>([&](auto Kk) {
            constexpr int k = Kk;
            if constexpr (K % k == 0 && fam_of(k, H) == K) {
                if ((ht >> (k - 1)) & 1u)
                    put_record(o.rec, slot++, o.cap, f, zz, k, 0u, lv[k - 1].x);
                if ((hb >> (k - 1)) & 1u)
                    put_record(o.rec, slot++, o.cap, f, -zz, k, 0u, lv[k - 1].y);
            }
        });
    }
}

// ---- staged kernel ---------------------------------------------------------------

// Shared-memory layout of family K over TB bins: term h has a top and a
// bottom box of h rows by W(h) bins (the term's span floor(f h/K) over the
// tile plus the slack of its 16-byte aligned start), each at a 128-byte
// boundary.
template <int TB, int K>
struct HGeom {
    static constexpr int W(int h) { return round_up(((TB - 1) * h + K - 1) / K + 4, 4); }
    static constexpr int BOX(int h) { return W(h) * h * 4; }
    static constexpr int TOP(int h)
    {
        int o = 0;
        for (int i = 1; i < h; ++i)
            o += 2 * round_up(BOX(i), 128);
        return o;
    }
    static constexpr int BOT(int h) { return TOP(h) + round_up(BOX(h), 128); }
    static constexpr int SMEM = TOP(K + 1);
    static constexpr uint32_t TX()
    {
        uint32_t b = 0;
        for (int h = 1; h <= K; ++h)
            b += 2u * (uint32_t)BOX(h);
        return b;
    }
};

template <int H, int K>
struct HStagedParams {
    CUtensorMap maps[K]; // term h: box (W(h), h) over the plane
    LevelBounds<H> lb;
    HitSink o;
    long long f_lo, f_hi;
    const uint32_t *order; // tile order over the plane, or null (linear)
};

// One CTA per tile of TB bins and row block j (pairs jK .. jK + K - 1); the
// grid runs every tile of block 0 first, then of block 1, ..., so the rows
// read at any one time are few and L2 holds them across the family's terms.
// ZG groups of TB threads share the block's boxes: group g walks the steps
// i = g, g + ZG, ... of the block, so a tile's shared memory serves ZG times
// the warps.  The step loop runs at run time (one step's code, so the
// instruction cache holds the kernel); the row offset of term h at step i,
// floor(i h/K) * W(h) * 4 bytes, comes from a table the CTA writes first,
// four terms per 16-byte load.
template <int H, int TB, int K, int ZG>
__global__ void __launch_bounds__(TB *ZG, 1024 / (TB * ZG)) hfrac_staged_kernel(const __grid_constant__ HStagedParams<H, K> p)
{
    using G = HGeom<TB, K>;
    constexpr int KQ = (K + 3) & ~3; // table row stride
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_storage;
    __shared__ __align__(16) int s_rw[K * KQ];
    const uint32_t sbase = smem_addr(smem);
    const uint32_t bar = smem_addr(&bar_storage);
    const int Z = (p.o.nt - 1) / 2;
    const int j = (int)blockIdx.y;
    const long long tile = p.order ? (long long)__ldg(p.order + blockIdx.x) : (long long)blockIdx.x;
    const unsigned F = (unsigned)(p.f_lo + tile * TB);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, G::TX());
        static_for<1, K + 1>([&](auto Hh) {
            constexpr int h = Hh;
            const int x = (int)((F * (unsigned)h) / (unsigned)K) & ~3;
            tma_load_2d(sbase + G::TOP(h), &p.maps[h - 1], x, Z + j * h, bar);
            tma_load_2d(sbase + G::BOT(h), &p.maps[h - 1], x, Z - j * h - h + 1, bar);
        });
    }
    for (int e = (int)threadIdx.x; e < K * KQ; e += TB * ZG) {
        const int i = e / KQ, h = e % KQ + 1;
        const int w = round_up(((TB - 1) * h + K - 1) / K + 4, 4);
        s_rw[e] = h <= K ? (i * h) / K * w * 4 : 0;
    }
    const unsigned f = F + threadIdx.x % TB;
    const int grp = (int)(threadIdx.x / TB); // warp-uniform (TB is a multiple of 32)
    const bool valid = (long long)f < p.f_hi;
    // this thread's column (bytes) in term h's boxes
    int col[K];
    static_for<1, K + 1>([&](auto Hh) {
        constexpr int h = Hh;
        const unsigned x = ((F * (unsigned)h) / (unsigned)K) & ~3u;
        col[h - 1] = (int)(4u * ((f * (unsigned)h) / (unsigned)K - x));
    });
    __syncthreads(); // the barrier and the table are ready before anyone reads them
    if (!__syncthreads_and(mbar_wait_bounded(bar, 0u, kWaitLimitNs))) {
        if (threadIdx.x == 0)
            set_status(p.o.counters, HS_ERR_TIMEOUT);
        mbar_wait_bounded(bar, 0u, kWaitLimitNs); // let copies in flight land
        return;
    }
    const int n_steps = min(K, Z - j * K + 1);
#pragma unroll 1
    for (int i = grp; i < n_steps; i += ZG) { // uniform over the group
        const int4 *rw = reinterpret_cast<const int4 *>(s_rw + i * KQ);
        float2 t[K];
        static_for<0, KQ / 4>([&](auto Qq) {
            constexpr int q = Qq;
            const int4 v = rw[q];
            const int o[4] = {v.x, v.y, v.z, v.w};
            static_for<0, 4>([&](auto Cc) {
                constexpr int h = 4 * q + Cc + 1;
                if constexpr (h <= K) {
                    const int at = G::TOP(h) + col[h - 1] + o[Cc];
                    const int ab = G::BOT(h) + (h - 1) * G::W(h) * 4 + col[h - 1] - o[Cc];
                    if (kCheck && (at < G::TOP(h) || at >= G::TOP(h) + G::BOX(h) ||
                                   ab < G::BOT(h) || ab >= G::BOT(h) + G::BOX(h))) {
                        set_status(p.o.counters, HS_ERR_BOUNDS);
                        t[h - 1] = make_float2(0.f, 0.f);
                    } else {
                        t[h - 1].x = *reinterpret_cast<const float *>(smem + at);
                        t[h - 1].y = *reinterpret_cast<const float *>(smem + ab);
                    }
                }
            });
        });
        family_levels<H, K>(t, j * K + i, f, valid, p.lb, p.o);
    }
}

template <int H, int TB, int K>
cudaError_t launch_staged_family(const HfracStagedLaunch &L, const CUtensorMap *maps,
                                 cudaStream_t s)
{
    using G = HGeom<TB, K>;
    constexpr int SMEM = G::SMEM;
    constexpr int ZG = 4; // row groups per tile
    static_assert(SMEM <= 227 * 1024, "family boxes exceed shared memory");
    static_assert(G::W(K) <= 256, "box wider than a TMA box");
    // set on every launch (as for the stretch kernel): the attribute belongs
    // to the current device's context
    const cudaError_t attr = cudaFuncSetAttribute(
        hfrac_staged_kernel<H, TB, K, ZG>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (attr != cudaSuccess)
        return attr;
    HStagedParams<H, K> p;
    std::memcpy(p.maps, maps, sizeof(CUtensorMap) * K);
    for (int k = 0; k < H; ++k)
        p.lb.lmin[k] = L.lmin ? L.lmin[k] : -__builtin_huge_valf();
    p.o = HitSink{L.ta, L.rec, L.counters, L.cap, L.nt};
    p.f_lo = L.f_lo;
    p.f_hi = L.f_hi;
    p.order = L.order;
    const long long n_tiles = (L.f_hi - L.f_lo + TB - 1) / TB;
    const int nblk = (L.nt - 1) / 2 / K + 1;
    hfrac_staged_kernel<H, TB, K, ZG>
        <<<dim3((unsigned)n_tiles, (unsigned)nblk), TB * ZG, SMEM, s>>>(p);
    return cudaGetLastError();
}

// Descriptors of every (family, term) box of one plane, heads in descending
// order, terms ascending: the family with head K starts at the sum of the
// larger heads.
template <int H, int TB>
CUresult encode_all(const HfracStagedLaunch &L, std::vector<CUtensorMap> &maps)
{
    maps.clear();
    CUresult r = CUDA_SUCCESS;
    static_for_host<0, n_heads(H)>([&](auto Ii) {
        constexpr int K = head_at(Ii, H);
        for (int h = 1; h <= K && r == CUDA_SUCCESS; ++h) {
            CUtensorMap m;
            r = encode_tensor_map(&m, HS_F32, L.fop, L.n, L.ld, L.nt, HGeom<TB, K>::W(h), h);
            maps.push_back(m);
        }
    });
    return r;
}

struct MapCache {
    const void *fop = nullptr;
    long long n = 0, ld = 0;
    int nt = 0, H = 0, tb = 0;
    std::vector<CUtensorMap> maps;
};
constexpr int kMapCacheSlots = 4;

template <int H, int TB>
cudaError_t launch_staged_all(const HfracStagedLaunch &L, cudaStream_t s, int *launches)
{
    // the descriptors of the last few planes, per host thread (equal address
    // and layout give equal descriptors; a run encodes only a plane it has
    // not seen, replacing the oldest entry)
    thread_local MapCache caches[kMapCacheSlots];
    thread_local int next_slot = 0;
    MapCache *hit = nullptr;
    for (MapCache &c : caches)
        if (c.fop == L.fop && c.n == L.n && c.ld == L.ld && c.nt == L.nt && c.H == H &&
            c.tb == TB)
            hit = &c;
    if (!hit) {
        MapCache &c = caches[next_slot];
        next_slot = (next_slot + 1) % kMapCacheSlots;
        c.fop = nullptr;
        if (encode_all<H, TB>(L, c.maps) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
        c.fop = L.fop;
        c.n = L.n;
        c.ld = L.ld;
        c.nt = L.nt;
        c.H = H;
        c.tb = TB;
        hit = &c;
    }
    MapCache &cache = *hit;
    cudaError_t e = cudaSuccess;
    int first = 0;
    static_for_host<0, n_heads(H)>([&](auto Ii) {
        constexpr int K = head_at(Ii, H);
        if (e == cudaSuccess) {
            e = launch_staged_family<H, TB, K>(L, cache.maps.data() + first, s);
            if (e == cudaSuccess)
                ++*launches;
        }
        first += K;
    });
    return e;
}

// ---- gather kernel ---------------------------------------------------------------

constexpr int kThreads = 128;
constexpr int kMaxPairsPerBlock = 64;

// One family K over this CTA's bins and row pairs [zz_lo, zz_hi].
template <int H, int K>
__device__ __forceinline__ void gather_family(const GenericArgs &a, const LevelBounds<H> &lb,
                                              long long *s_off, unsigned f, bool valid,
                                              int zz_lo, int zz_hi)
{
    constexpr int KP = (K + 1) & ~1; // table row stride: pairs of offsets per 16 bytes
    const int Z = (a.nt - 1) / 2;
    const int n_zz = zz_hi - zz_lo + 1;
    for (int i = threadIdx.x; i < n_zz * KP; i += kThreads) {
        const unsigned zz = (unsigned)(zz_lo + i / KP), h = (unsigned)(i % KP) + 1u;
        s_off[i] = (long long)((zz * h) / (unsigned)K) * a.ld * (long long)sizeof(float);
    }
    __syncthreads();

    const HitSink o{a.ta, a.rec, a.counters, a.cap, a.nt};
    const char *plane_lo = static_cast<const char *>(a.fop);
    const char *plane_hi =
        plane_lo + ((long long)(a.nt - 1) * a.ld + a.n) * (long long)sizeof(float);
    uint32_t *a_counters = a.counters;
    // this family's bin offsets in the centre row, once per thread
    const char *pc = reinterpret_cast<const char *>(static_cast<const float *>(a.fop) +
                                                    (long long)Z * a.ld);
    const char *tp[K];
    static_for<1, K + 1>([&](auto Hh) {
        constexpr int h = Hh;
        tp[h - 1] = pc + sizeof(float) * ((f * (unsigned)h) / (unsigned)K);
    });
    for (int zl = 0; zl < n_zz; ++zl) { // uniform over the CTA
        const longlong2 *d2 = reinterpret_cast<const longlong2 *>(s_off + zl * KP);
        float2 t[K];
        // plane value at byte address a (checked builds: inside the plane)
        auto ld = [&](const char *a) -> float {
            if (kCheck && (a < plane_lo || a >= plane_hi)) {
                set_status(a_counters, HS_ERR_BOUNDS);
                return 0.f;
            }
            return __ldg(reinterpret_cast<const float *>(a));
        };
        static_for<0, KP / 2>([&](auto Ii) {
            constexpr int i = Ii;
            const longlong2 d = d2[i];
            t[2 * i] = make_float2(ld(tp[2 * i] + d.x), ld(tp[2 * i] - d.x));
            if constexpr (2 * i + 1 < K)
                t[2 * i + 1] = make_float2(ld(tp[2 * i + 1] + d.y), ld(tp[2 * i + 1] - d.y));
        });
        family_levels<H, K>(t, zz_lo + zl, f, valid, lb, o);
    }
}

template <int H>
__global__ void __launch_bounds__(kThreads)
    hfrac_pair_kernel(const GenericArgs a, const LevelBounds<H> lb, int pairs_per_block)
{
    __shared__ __align__(16) long long s_off[kMaxPairsPerBlock * ((H + 1) & ~1)];
    const int Z = (a.nt - 1) / 2;
    const long long f64 = a.f_lo + (long long)blockIdx.x * kThreads + threadIdx.x;
    const bool valid = f64 < a.f_hi;
    const unsigned f = (unsigned)(valid ? f64 : a.f_lo);
    const int zz_lo = (int)blockIdx.y * pairs_per_block;
    const int zz_hi = min(Z, zz_lo + pairs_per_block - 1);
    static_for<0, n_heads(H)>([&](auto Ii) {
        constexpr int i = Ii;
        if (blockIdx.z == (unsigned)i)
            gather_family<H, head_at(i, H)>(a, lb, s_off, f, valid, zz_lo, zz_hi);
    });
}

template <int H>
cudaError_t launch_gather(const GenericArgs &a, const float *lmin_host, cudaStream_t s)
{
    LevelBounds<H> lb;
    for (int k = 0; k < H; ++k)
        lb.lmin[k] = lmin_host ? lmin_host[k] : -__builtin_huge_valf();
    const long long nbins = a.f_hi - a.f_lo;
    const long long bx = (nbins + kThreads - 1) / kThreads;
    const int pairs = (a.nt - 1) / 2 + 1;
    constexpr int nf = n_heads(H);
    // enough CTAs to fill the GPU several times over: split the row pairs,
    // but keep at least 8 pairs per CTA so the offset table pays for itself
    const long long want = (4 * 152 * 8 + bx * nf - 1) / (bx * nf);
    int ppb = (int)std::max(1LL, (pairs + want - 1) / want);
    ppb = std::min(kMaxPairsPerBlock, std::max(ppb, std::min(pairs, 8)));
    const int by = (pairs + ppb - 1) / ppb;
    hfrac_pair_kernel<H><<<dim3((unsigned)bx, (unsigned)by, (unsigned)nf), kThreads, 0, s>>>(
        a, lb, ppb);
    return cudaGetLastError();
}

} // namespace

bool hfrac_pairs_available(const GenericArgs &a)
{
    return a.dtype == HS_F32 && a.index == HS_INDEX_HFRAC && a.zround == HS_ZROUND_SYMMETRIC &&
           (a.H == 8 || a.H == 16) && a.f_hi <= (1LL << 31) / a.H &&
           (a.f_hi - a.f_lo + kThreads - 1) / kThreads <= 0x7fffffffLL;
}

cudaError_t launch_hfrac_pairs(const GenericArgs &a, const float *lmin_host, cudaStream_t s)
{
    if (a.f_hi <= a.f_lo)
        return cudaSuccess;
    return a.H == 8 ? launch_gather<8>(a, lmin_host, s) : launch_gather<16>(a, lmin_host, s);
}

bool hfrac_staged_available(int nt, long long n, long long ld, int H, int dtype, int index,
                            int zround, int tb)
{
    return dtype == HS_F32 && index == HS_INDEX_HFRAC && zround == HS_ZROUND_SYMMETRIC &&
           (H == 8 || H == 16) && (tb == 64 || tb == 128) && (ld * 4) % 16 == 0 &&
           n + tb <= (1LL << 31) / H && nt >= 1 && nt <= 32767;
}

cudaError_t launch_hfrac_staged(const HfracStagedLaunch &L, cudaStream_t s, int *launches)
{
    if (L.f_hi <= L.f_lo)
        return cudaSuccess;
    if (L.H == 8)
        return L.tb == 64 ? launch_staged_all<8, 64>(L, s, launches)
                          : launch_staged_all<8, 128>(L, s, launches);
    return L.tb == 64 ? launch_staged_all<16, 64>(L, s, launches)
                      : launch_staged_all<16, 128>(L, s, launches);
}

} // namespace hs
