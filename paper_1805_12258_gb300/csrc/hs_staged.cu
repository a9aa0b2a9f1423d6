// hs_staged.cu -- the staged harmonic-summing kernel (the hot path).
//
// One CTA owns an output tile of TB consecutive bins [f0, f0+TB) x all NT
// template rows.  For each stretch factor m = 1..H (Eq. 1) the tile reads the
// input span rows [Z - Z/m, Z + Z/m] x bins [floor(f0/m), floor((f0+TB-1)/m)];
// one elected thread stages every span into shared memory with one 2-D TMA
// box per m, all completing on a single mbarrier, so each plane point crosses
// HBM about once per tile that needs it (the "load the necessary points of a
// chunk" idea of Section IV-C2, with TMA boxes instead of the paper's
// reordered plane).
//
// Each thread then owns one bin f and all NT rows of the tile.  Rows are
// walked outward from z = 0 as mirrored pairs (+zz, -zz): under the
// symmetric rounding rho(z, m) = sign(z) floor(|z|/m) the two rows of a pair
// change their source row for the same m, so the values of all m stay in
// registers and are reloaded from shared memory only when m divides zz.  The
// pair's H cumulative sums of Eq. 2 are formed with packed FP32 adds
// (add.rn.f32x2), in ascending m -- the order of Eq. 2, so every sum is the
// same FP32 number as a plain scalar loop.
//
// Detection uses an exact two-stage test.  With non-negative inputs a level
// sum never decreases with k, so "no level in [a, b] exceeds its threshold"
// follows from HP_b <= min_{k in [a,b]} TA(k, row), and a fortiori from
// HP_b <= the smallest threshold of the group over all rows, which is the
// bound used (four values held in registers; per-row bounds would have to
// be re-read for every row and cost more than they save).  The fast pass tests only
// the level groups [1,2], [3,4], [5,8], [9,16] this way and marks the row pairs
// that might hold a hit; a slow pass recomputes those pairs level by level and
// appends the true hits (warp ballot + prefix, one atomic per warp).  A thread
// that loaded any value with its sign bit set (negative input, -0) sends all
// of its rows to the slow pass, so the result never depends on the inputs
// being non-negative.  For 16-bit planes the group thresholds are lowered by
// the storage error bound and the slow pass re-evaluates possible hits from
// the FP32 copy, so candidates match the FP32 path.
#include <cstring>
#include <mutex>

#include "hs_device.cuh"
#include "hs_internal.h"

namespace hs {
namespace {

constexpr int round_up(int x, int a) { return (x + a - 1) / a * a; }

// Level groups of the prefilter: a group ends at every power of two >= 2
// and at H.
constexpr bool group_end(int m, int H) { return m == H || (m >= 2 && (m & (m - 1)) == 0); }
constexpr int group_index(int m, int H)
{
    int g = 0;
    for (int i = 1; i < m; ++i)
        g += group_end(i, H) ? 1 : 0;
    return g;
}
constexpr int n_groups(int H) { return group_index(H, H) + 1; }

template <int NT, int H, int TB, typename T>
struct Cfg {
    static constexpr int Z = (NT - 1) / 2;
    static constexpr int ES = (int)sizeof(T);
    static constexpr int ALIGN = 16 / ES; // elements per 16 bytes (TMA x alignment)
    static constexpr int G = n_groups(H);
    static constexpr int R(int m) { return Z / m; }
    static constexpr int ROWS(int m) { return 2 * R(m) + 1; }
    // Box width: exact when every tile start f0/m is 16-byte aligned,
    // otherwise the widest span plus the alignment slack of its start.
    static constexpr int W(int m)
    {
        return (TB % (m * ALIGN) == 0) ? TB / m : round_up((TB - 1) / m + ALIGN + 1, ALIGN);
    }
    static constexpr int BYTES(int m) { return ROWS(m) * W(m) * ES; }
    static constexpr int OFF(int m)
    {
        int o = 0;
        for (int i = 1; i < m; ++i)
            o += round_up(BYTES(i), 128);
        return o;
    }
    static constexpr int SMEM = OFF(H + 1);
    static constexpr int TX()
    {
        int t = 0;
        for (int i = 1; i <= H; ++i)
            t += BYTES(i);
        return t;
    }
    static_assert(NT % 2 == 1, "odd template count");
    static_assert(Z <= 63, "row-pair mask is 64 bits");
    static_assert(H <= kMaxStagedH && G <= kMaxGroups, "level count");
    static_assert(TB <= 256 && TB % ALIGN == 0, "TMA box width");
    static_assert(TX() < (1 << 20), "mbarrier transaction count");
};

template <int NT, int H>
struct Params {
    CUtensorMap maps[H];    // one 2-D box per stretch factor m
    float tmin[n_groups(H)]; // prefilter threshold per level group (min over rows)
    const float *ta;        // exact thresholds [H][NT] (device)
    const float *fop32;     // FP32 copy for rechecks, or null
    const uint32_t *order;  // tile order (device) or null
    hs_cand *rec;
    uint32_t *counters;
    uint32_t cap;
    float delta;            // 16-bit storage relative error bound (0 for FP32)
    float band_abs;         // 16-bit storage absolute error bound
    long long n;
    int tile_lo;
};

// Level m value of the FP32 copy at (z, f): the Eq. 2 chain in FP32,
// ascending m, i.e. exactly the number the FP32 path computes.
__device__ float chain_f32(const float *fop32, int Z, long long n, int z, int f, int k)
{
    float s = 0.f;
    for (int m = 1; m <= k; ++m) {
        const int rho = z >= 0 ? z / m : -((-z) / m);
        const float v = __ldg(fop32 + (long long)(rho + Z) * n + f / m);
        s = (m == 1) ? v : s + v;
    }
    return s;
}

template <int NT, int H, int TB, typename T>
__global__ void __launch_bounds__(TB, 384 / TB) staged_kernel(const __grid_constant__ Params<NT, H> p)
{
    using C = Cfg<NT, H, TB, T>;
    constexpr int Z = C::Z;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_storage;

    const uint32_t bar = smem_addr(&bar_storage);
    const uint32_t sbase = smem_addr(smem);
    const int tid = threadIdx.x;
    const int slot = p.tile_lo + (int)blockIdx.x;
    const int tile = p.order ? (int)__ldg(p.order + slot) : slot;
    const int f0 = tile * TB;

    if (tid == 0) {
        static_for<0, H>([&](auto M) { prefetch_tmap(&p.maps[M]); });
        mbar_init(bar, 1);
    }
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(bar, (uint32_t)C::TX());
        static_for<1, H + 1>([&](auto M) {
            constexpr int m = M;
            const int x = (f0 / m) & ~(C::ALIGN - 1);
            tma_load_2d(sbase + C::OFF(m), &p.maps[m - 1], x, Z - C::R(m), bar);
        });
    }

    // This thread's column in every span, as an element index of the centre
    // row (template z = 0), computed while the copies are in flight.
    const int f = f0 + tid;
    const bool valid = (long long)f < p.n;
    const T *sm = reinterpret_cast<const T *>(smem);
    int bidx[H];
    static_for<0, H>([&](auto M) {
        constexpr int m = M + 1;
        const int col = f / m - ((f0 / m) & ~(C::ALIGN - 1));
        bidx[M] = C::OFF(m) / C::ES + C::R(m) * C::W(m) + col;
    });

    bool ok = mbar_wait_bounded(bar, 0, kWaitLimitNs);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) {
        if ((tid & 31) == 0)
            set_status(p.counters, HS_ERR_TIMEOUT);
        mbar_wait_bounded(bar, 0, kWaitLimitNs); // let copies in flight land
        return;
    }

    // ---- fast pass: all rows, group prefilter --------------------------------
    float tg[C::G];
    static_for<0, C::G>([&](auto g) { tg[g] = p.tmin[g]; });
    uint32_t negbits = 0u;
    uint64_t mask = 0ull;
    float2 cur[H];
    {
        float acc = 0.f;
        bool maybe = false;
        static_for<0, H>([&](auto M) {
            constexpr int m = M + 1;
            const float v = to_f32(sm[bidx[M]]);
            cur[M] = make_float2(v, v);
            negbits |= __float_as_uint(v);
            acc = (m == 1) ? v : acc + v;
            if constexpr (group_end(m, H))
                maybe |= !(acc <= tg[group_index(m, H)]);
        });
        mask = maybe ? 1ull : 0ull;
    }
    static_for<1, Z + 1>([&](auto ZZ) {
        constexpr int zz = ZZ;
        float2 acc = cur[0];
        bool maybe = false;
        static_for<0, H>([&](auto M) {
            constexpr int m = M + 1;
            if constexpr (zz % m == 0) {
                constexpr int off = (zz / m) * C::W(m);
                const float t = to_f32(sm[bidx[M] + off]);
                const float b = to_f32(sm[bidx[M] - off]);
                cur[M] = make_float2(t, b);
                negbits |= __float_as_uint(t) | __float_as_uint(b);
            }
            if constexpr (m == 1)
                acc = cur[0];
            else
                acc = __fadd2_rn(acc, cur[M]);
            if constexpr (group_end(m, H)) {
                maybe |= !(acc.x <= tg[group_index(m, H)]);
                maybe |= !(acc.y <= tg[group_index(m, H)]);
            }
        });
        if (maybe)
            mask |= 1ull << zz;
    });
    if (!valid)
        mask = 0ull;
    else if (negbits >> 31)
        mask = (Z == 63) ? ~0ull : ((1ull << (Z + 1)) - 1ull);

    // ---- slow pass: exact per-level test of the marked row pairs --------------
    // scan(z, write, slot): level sums of row z in Eq. 2 order; returns the hit
    // mask over levels and, when write is set, appends the records from slot.
    auto scan = [&](int z, bool write, uint32_t rslot) -> uint32_t {
        float acc = 0.f, ab = 0.f;
        uint32_t hits = 0u;
        static_for<0, H>([&](auto M) {
            constexpr int m = M + 1;
            const int rho = z >= 0 ? z / m : -((-z) / m);
            const float v = to_f32(sm[bidx[M] + rho * C::W(m)]);
            acc = (m == 1) ? v : acc + v;
            ab += fabsf(v);
            const float thr = __ldg(p.ta + M * NT + (z + Z));
            float power = acc;
            uint32_t flags = 0u;
            bool hit;
            if (p.delta == 0.f) {
                hit = acc > thr;
            } else if (p.fop32 != nullptr) {
                hit = false;
                if (!(acc == acc && acc + (p.delta * ab + p.band_abs) < thr)) {
                    power = chain_f32(p.fop32, Z, p.n, z, f, m);
                    hit = power > thr;
                }
            } else {
                hit = acc > thr;
                flags = HS_FLAG_LOWP |
                        (fabsf(acc - thr) <= p.delta * ab + p.band_abs ? HS_FLAG_NEAR : 0u);
            }
            if (hit) {
                hits |= 1u << M;
                if (write)
                    put_record(p.rec, rslot++, p.cap, (uint32_t)f, z, m, flags, power);
            }
        });
        return hits;
    };

    while (__any_sync(0xffffffffu, mask != 0ull)) {
        int zz = -1;
        if (mask != 0ull) {
            zz = __ffsll((long long)mask) - 1;
            mask &= mask - 1ull;
        }
        uint32_t ht = 0u, hb = 0u;
        if (zz >= 0) {
            ht = scan(zz, false, 0u);
            if (zz > 0)
                hb = scan(-zz, false, 0u);
        }
        uint32_t rs = warp_reserve(p.counters, (uint32_t)(__popc(ht) + __popc(hb)));
        if (ht)
            scan(zz, true, rs);
        if (hb)
            scan(-zz, true, rs + (uint32_t)__popc(ht));
    }
}

template <int NT, int H, int TB, typename T>
cudaError_t launch_one(const StagedLaunch &a, cudaStream_t s)
{
    using C = Cfg<NT, H, TB, T>;
    Params<NT, H> p;
    std::memset(&p, 0, sizeof p);
    std::memcpy(p.maps, a.maps, sizeof(CUtensorMap) * H);
    for (int g = 0; g < C::G; ++g)
        p.tmin[g] = a.tmin_host[g];
    p.ta = a.ta;
    p.fop32 = a.fop32;
    p.order = a.order;
    p.rec = a.rec;
    p.counters = a.counters;
    p.cap = a.cap;
    p.delta = a.delta;
    p.band_abs = a.band_abs;
    p.n = a.n;
    p.tile_lo = a.tile_lo;
    auto kern = staged_kernel<NT, H, TB, T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         C::SMEM);
    if (e != cudaSuccess)
        return e;
    const int tiles = a.tile_hi - a.tile_lo;
    if (tiles <= 0)
        return cudaSuccess;
    kern<<<tiles, TB, C::SMEM, s>>>(p);
    return cudaGetLastError();
}

// Shapes compiled into the library: the SKA plane (85 templates, 16 levels),
// the small plane (21 templates, 8 levels), each for FP32, BF16 and FP16
// storage; tile widths 64/128/256 for the FP32 SKA shape (autotuner choices).
#define HS_STAGED_SHAPES(X)                                                                   \
    X(85, 16, 128, float, HS_F32)                                                             \
    X(85, 16, 64, float, HS_F32)                                                              \
    X(85, 16, 256, float, HS_F32)                                                             \
    X(85, 16, 128, __nv_bfloat16, HS_BF16)                                                    \
    X(85, 16, 128, __half, HS_F16)                                                            \
    X(21, 8, 128, float, HS_F32)                                                              \
    X(21, 8, 128, __nv_bfloat16, HS_BF16)                                                     \
    X(21, 8, 128, __half, HS_F16)

template <int NT, int H, int TB, typename T>
void box_of(int m, int *w, int *rows)
{
    *w = Cfg<NT, H, TB, T>::W(m);
    *rows = Cfg<NT, H, TB, T>::ROWS(m);
}

} // namespace

bool staged_available(const StagedShape &sh)
{
#define X(NT_, H_, TB_, T_, DT_)                                                                   \
    if (sh.nt == NT_ && sh.H == H_ && sh.tb == TB_ && sh.dtype == DT_)                           \
        return true;
    HS_STAGED_SHAPES(X)
#undef X
    return false;
}

int staged_smem_bytes(const StagedShape &sh)
{
#define X(NT_, H_, TB_, T_, DT_)                                                                   \
    if (sh.nt == NT_ && sh.H == H_ && sh.tb == TB_ && sh.dtype == DT_)                           \
        return Cfg<NT_, H_, TB_, T_>::SMEM;
    HS_STAGED_SHAPES(X)
#undef X
    return -1;
}

void staged_box(const StagedShape &sh, int m, int *width, int *rows)
{
    *width = *rows = 0;
#define X(NT_, H_, TB_, T_, DT_)                                                                   \
    if (sh.nt == NT_ && sh.H == H_ && sh.tb == TB_ && sh.dtype == DT_) {                         \
        box_of<NT_, H_, TB_, T_>(m, width, rows);                                                 \
        return;                                                                               \
    }
    HS_STAGED_SHAPES(X)
#undef X
}

int staged_groups(int H, int *ends)
{
    int g = 0;
    for (int m = 1; m <= H; ++m)
        if (group_end(m, H))
            ends[g++] = m;
    return g;
}

cudaError_t launch_staged(const StagedLaunch &a, cudaStream_t s)
{
    const StagedShape &sh = a.sh;
#define X(NT_, H_, TB_, T_, DT_)                                                                   \
    if (sh.nt == NT_ && sh.H == H_ && sh.tb == TB_ && sh.dtype == DT_)                           \
        return launch_one<NT_, H_, TB_, T_>(a, s);
    HS_STAGED_SHAPES(X)
#undef X
    return cudaErrorInvalidValue;
}

} // namespace hs
