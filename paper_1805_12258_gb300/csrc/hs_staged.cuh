// hs_staged.cuh -- the staged harmonic-summing kernel (the hot path): device
// code and launch templates.  Each hs_k_*.cu file instantiates the shapes
// of one family and registers their entry points (hs_shapes.h); hs_staged.cu
// dispatches a plan, batch or launch to its shape.
//
// Work unit: a tile of TB consecutive bins [f0, f0+TB) x all NT template
// rows, one CTA of TB threads; thread t owns bin f = f0 + t and every row.
// For each stretch factor m = 1..H (Eq. 1) the tile reads the input span
// rows [Z - Z/m, Z + Z/m] x bins [floor(f0/m), floor((f0+TB-1)/m)] -- the
// "necessary points" of the chunk (Section IV-C2), gathered with 2-D TMA
// boxes instead of the paper's reordered plane -- so each plane point crosses
// HBM about once per tile that needs it.  One elected thread issues one box
// per m, all completing on a single mbarrier; or, on FP32 planes declared
// non-negative, level 1 in three row bands: the centre rows [Z - Z/2, Z + Z/2]
// complete with the spans of m >= 2 (whose rows all lie in that band) on one
// mbarrier, the outer rows on a second that the walk waits for only when it
// reaches pair Z/2 + 1, so summing starts before the outer rows land.
//
// Rows are walked outward from z = 0 as mirrored pairs (+zz, -zz).  Under the
// symmetric rounding rho(z, m) = sign(z) floor(|z|/m) both rows of a pair
// change their source row for the same m, so the values of all m stay in
// registers and are reloaded from shared memory only when m divides zz.
//
// Detection is exact in two stages.  With non-negative inputs a level sum
// never decreases with k, so "no level in [a, b] exceeds its threshold"
// follows from HP_b <= min over the group's levels and all rows of TA, the
// group bound (a few values in registers; per-row bounds would have to be
// re-read for every row and cost more than they save).  The fast pass forms
// HP_b only at the group ends (each group summed as a tree with packed FP32
// adds over the pair, kept from pair to pair and re-added only where one of
// its levels was reloaded; each group's bound rides in the value of its last
// level, so a group's test is the sign of the running sum, the bounds lowered
// by the FP32 error of that order) and marks the row pairs that might hold a
// hit; the slow pass recomputes those rows
// level by level in ascending m (the order of Eq. 2) and appends the true
// hits with warp ballot + prefix and one atomic per warp.  A thread that
// loaded any value with its sign bit set (a negative input or -0) sends all
// its rows to the slow pass, so the result never depends on the inputs being
// non-negative.  For 16-bit planes the bounds are lowered by the storage
// error too and the slow pass re-evaluates possible hits from the FP32 copy,
// so candidates match the FP32 path record for record.
//
// Kernels: staged_kernel (one plane; one CTA per tile, or resident CTAs
// walking the tile order), pipe_kernel (one plane; a persistent CTA per SM
// with a producer warp and a ring of stages), batched_kernel (many planes,
// descriptors in the launch's parameter block).
#pragma once

#include <algorithm>
#include <cstring>

#include "hs_device.cuh"
#include "hs_internal.h"
#include "hs_shapes.h"

namespace hs {
namespace {

constexpr int round_up(int x, int a) { return (x + a - 1) / a * a; }
constexpr int cmin(int a, int b) { return a < b ? a : b; }

// Level groups of the prefilter: a group ends at 2, 4, 8, then every 4
// levels, and at H.
constexpr bool group_end(int m, int H)
{
    return m == H || m == 2 || m == 4 || (m >= 8 && m % 4 == 0);
}
constexpr int group_index(int m, int H)
{
    int g = 0;
    for (int i = 1; i < m; ++i)
        g += group_end(i, H) ? 1 : 0;
    return g;
}
constexpr int n_groups(int H) { return group_index(H, H) + 1; }
// True when some level m in [lo, hi] changes its source row at pair zz >= 1
// (m divides zz), i.e. when the walk reloads it there.
constexpr bool reloads_any(int zz, int lo, int hi)
{
    for (int m = lo; m <= hi; ++m)
        if (zz % m == 0)
            return true;
    return false;
}

template <int NT, int H, int TB, typename T>
struct Cfg {
    static constexpr int Z = (NT - 1) / 2;
    static constexpr int ES = (int)sizeof(T);
    static constexpr int ALIGN = 16 / ES; // elements per 16 bytes (TMA x alignment)
    static constexpr int G = n_groups(H);
    // first and last level of prefilter group g
    static constexpr int GHI(int g)
    {
        for (int m = 1, i = 0; m <= H; ++m)
            if (group_end(m, H) && i++ == g)
                return m;
        return H;
    }
    static constexpr int GLO(int g) { return g == 0 ? 1 : GHI(g - 1) + 1; }
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
    // Level 1 split in row bands: the centre rows [Z - RB, Z + RB] (every
    // row the pairs zz <= RB read, with all spans m >= 2, whose rows lie
    // within Z/2 of the centre) and the outer rows (OUT on each side).
    static constexpr int RB = Z / 2;
    static constexpr int OUT = Z - RB;
    static constexpr int BYTES_CENTRE = (2 * RB + 1) * W(1) * ES;
    static constexpr int BYTES_OUTER = OUT * W(1) * ES;
    static constexpr int TX_CENTRE() { return TX() - BYTES(1) + BYTES_CENTRE; }
    // CTAs that fit on an SM by shared memory (228 KB, 1 KB reserved per
    // CTA), at most 8
    static constexpr int CTAS_SMEM = cmin(8, 233472 / (SMEM + 1024 + 64));
    static constexpr int TX()
    {
        int t = 0;
        for (int i = 1; i <= H; ++i)
            t += BYTES(i);
        return t;
    }
    static_assert(NT % 2 == 1, "odd template count");
    static_assert(Z <= 63, "row-pair mask is 64 bits");
    static_assert(H >= 2 && H <= kMaxStagedH && G <= kMaxGroups, "level count");
    static_assert(TB <= 256 && TB % ALIGN == 0 && TB % 32 == 0, "TMA box width, whole warps");
    static_assert(TX() < (1 << 20), "mbarrier transaction count");
};

template <int NT, int H, typename T>
struct Params {
    CUtensorMap maps[H];    // one 2-D box per stretch factor m (its whole span)
    CUtensorMap split1[2];  // level 1 in bands: centre rows, one outer side
    float tmin[n_groups(H)]; // prefilter bound per level group (min over rows)
    const float *ta;        // exact thresholds [H][NT] (device)
    const float *fop32;     // FP32 copy for rechecks, or null
    const uint32_t *order;  // tile order (device) or null
    hs_cand *rec;
    uint32_t *counters;
    uint32_t cap;
    float delta;            // 16-bit storage relative error bound (0 for FP32)
    float band_abs;         // 16-bit storage absolute error bound
    long long n;
    long long ld;           // row pitch of the FP32 copy (elements)
    int tile_lo;            // first slot of the tile order this launch covers
    int n_slots;            // tiles of this launch
    int nt_rt;              // templates of the plane (<= NT; kernels with runtime rows)
    uint2 *pend;            // 16-bit planes with an FP32 copy: marked row pairs
    uint32_t *pend_count;   // (bin, pair) for the recheck kernel, or null
    uint32_t pend_cap;
};

// Opt-in bounds checks (-DHS_CHECK_BOUNDS).  A checked build tests every
// shared-memory read of the walk and the exact pass against its own level's
// span in the stage (and each thread's column against the span's width), and
// every global read of the exact pass against its threshold table or plane;
// an index outside sets HS_ERR_BOUNDS in the status word and the read is
// skipped (0 for a value, +inf for a threshold).  Never a trap.
#ifdef HS_CHECK_BOUNDS
constexpr bool kCheckBounds = true;
#else
constexpr bool kCheckBounds = false;
#endif

// Pairwise (tree) sum of cur[LO..HI] with packed adds; depth log2(HI-LO+1).
template <int LO, int HI, int N>
__device__ __forceinline__ float2 tree_sum(const float2 (&cur)[N])
{
    if constexpr (LO == HI) {
        return cur[LO];
    } else {
        constexpr int MID = (LO + HI) / 2;
        return __fadd2_rn(tree_sum<LO, MID>(cur), tree_sum<MID + 1, HI>(cur));
    }
}

// What one tile reads and writes: its plane's descriptors and size, and the
// candidate buffer its hits go to (one plane for hs_run, a beam of a batch).
struct TileTarget {
    const CUtensorMap *maps; // H descriptors (parameter or global space)
    const CUtensorMap *split1; // level-1 band descriptors (centre, outer), or null
    const float *fop32;      // FP32 copy for rechecks (row pitch ld), or null
    long long n;             // bins of the plane
    long long ld;            // row pitch of the FP32 copy, in elements
    hs_cand *rec;
    uint32_t *counters;
    uint32_t cap;
    int zr;                  // runtime-row kernels: the plane's Z = (templates - 1) / 2
    int nt;                  // runtime-row kernels: the plane's template count
    uint2 *pend;             // pending list of marked row pairs (bin, pair) that the
    uint32_t *pend_count;    // recheck kernel decides from the FP32 copy; null: the
    uint32_t pend_cap;       // exact pass decides them in the tile
};

// Issue the H boxes of the tile starting at bin f0 into the stage (thread 0).
// xoff: the bin of the plane's descriptors at which this plane starts (a
// beam of a packed batch; 0 otherwise), a multiple of 16 bytes.
// RT: the plane has tt.nt <= NT templates; each box keeps the height of
// the compiled shape, centred on the plane's centre row tt.zr, and the rows
// outside the plane arrive as zeros (TMA fills out-of-range coordinates) and
// are never read.
template <int NT, int H, int TB, typename T, bool RT = false>
__device__ __forceinline__ void issue_tile(const TileTarget &tt, int f0, uint32_t sbase,
                                           uint32_t bar, int xoff = 0)
{
    using C = Cfg<NT, H, TB, T>;
    const int zc = RT ? tt.zr : C::Z;
    mbar_arrive_expect_tx(bar, (uint32_t)C::TX());
    static_for<1, H + 1>([&](auto M) {
        constexpr int m = M;
        const int x = xoff + ((f0 / m) & ~(C::ALIGN - 1));
        tma_load_2d(sbase + C::OFF(m), &tt.maps[m - 1], x, zc - C::R(m), bar);
    });
}

// Issue the tile's boxes with level 1 in bands (thread 0): the centre band
// and the spans m >= 2 complete on `bar`, the two outer bands on `bar_out`.
template <int NT, int H, int TB, typename T>
__device__ __forceinline__ void issue_tile_banded(const TileTarget &tt, int f0, uint32_t sbase,
                                                  uint32_t bar, uint32_t bar_out, int xoff = 0)
{
    using C = Cfg<NT, H, TB, T>;
    constexpr int ROWB = C::W(1) * C::ES; // bytes per level-1 row in shared memory
    const int x1 = xoff + f0;
    mbar_arrive_expect_tx(bar, (uint32_t)C::TX_CENTRE());
    tma_load_2d(sbase + (C::Z - C::RB) * ROWB, &tt.split1[0], x1, C::Z - C::RB, bar);
    static_for<2, H + 1>([&](auto M) {
        constexpr int m = M;
        const int x = xoff + ((f0 / m) & ~(C::ALIGN - 1));
        tma_load_2d(sbase + C::OFF(m), &tt.maps[m - 1], x, C::Z - C::R(m), bar);
    });
    mbar_arrive_expect_tx(bar_out, (uint32_t)(2 * C::BYTES_OUTER));
    tma_load_2d(sbase, &tt.split1[1], x1, 0, bar_out);
    tma_load_2d(sbase + (C::Z + C::RB + 1) * ROWB, &tt.split1[1], x1, C::Z + C::RB + 1, bar_out);
}

// Wait for the tile's stage (phase `parity` of `bar`), run the fast pass and
// the slow pass, append the hits to tt's buffer.  Called by every thread of
// the CTA; returns false (CTA-uniformly) if the stage did not arrive in time.
// any_of(v) returns the OR of v over the threads that sum the tile (the CTA,
// or one consumer group of the pipelined kernel) and synchronises them.
struct CtaOr {
    __device__ __forceinline__ bool operator()(bool v) const { return __syncthreads_or(v) != 0; }
};

// SIGNCHK: watch every loaded value's sign bit and send a thread that saw one
// set to the exact pass (off only when the caller declares the plane
// non-negative).
// BANDED: level 1's outer rows complete on bar_out, waited for only when the
// walk reaches them (pair RB + 1).
// RT: runtime rows (tt.nt <= NT templates, centre row tt.zr): the walk
// records pairs past tt.zr as clear and the thresholds are indexed by the
// plane's own template count.
template <int NT, int H, int TB, typename T, typename P, typename AnyOf = CtaOr,
          bool SIGNCHK = true, bool BANDED = false, bool RT = false>
__device__ __forceinline__ bool sum_tile(const P &p, const TileTarget &tt,
                                         int f0, const unsigned char *smem, uint32_t bar,
                                         uint32_t parity, AnyOf any_of = AnyOf{},
                                         uint32_t bar_out = 0u)
{
    using C = Cfg<NT, H, TB, T>;
    constexpr int Z = C::Z;
    static_assert(!(RT && BANDED), "runtime rows use one barrier");
    const int zr = RT ? tt.zr : Z;    // the plane's centre row
    const int ntr = RT ? tt.nt : NT;  // the plane's template count (threshold stride)
    const int tid = (int)threadIdx.x % TB;

    // This thread's column in every span, as an element index of the centre
    // row (template z = 0), computed while the copies are in flight.
    const int f = f0 + tid;
    const bool valid = (long long)f < tt.n;
    const T *sm = reinterpret_cast<const T *>(smem);
    int bidx[H];
    static_for<0, H>([&](auto M) {
        constexpr int m = M + 1;
        const int col = f / m - ((f0 / m) & ~(C::ALIGN - 1));
        bidx[M] = C::OFF(m) / C::ES + C::R(m) * C::W(m) + col;
        if constexpr (kCheckBounds) {
            if (col < 0 || col >= C::W(m))
                set_status(tt.counters, HS_ERR_BOUNDS);
        }
    });
    // level m's value at element idx of the stage (checked builds: inside
    // level m's own span, else skipped)
    auto sld = [&](auto M, int idx) -> float {
        if constexpr (kCheckBounds) {
            constexpr int m = decltype(M)::value + 1;
            constexpr int lo = C::OFF(m) / C::ES, hi = lo + C::ROWS(m) * C::W(m);
            if (idx < lo || idx >= hi) {
                set_status(tt.counters, HS_ERR_BOUNDS);
                return 0.f;
            }
        }
        return to_f32(sm[idx]);
    };
    // threshold of level M + 1 for row z (checked builds: inside the table)
    auto thr_of = [&](auto M, int z) -> float {
        if constexpr (kCheckBounds) {
            if (z + zr < 0 || z + zr >= ntr) {
                set_status(tt.counters, HS_ERR_BOUNDS);
                return __int_as_float(0x7f800000);
            }
        }
        return __ldg(p.ta + decltype(M)::value * ntr + (z + zr));
    };
    // the FP32 copy at (row rho of the plane's centre-relative rows, bin b)
    auto copy_at = [&](int rho, int b) -> float {
        if constexpr (kCheckBounds) {
            if (rho + zr < 0 || rho + zr >= ntr || b < 0 || (long long)b >= tt.n) {
                set_status(tt.counters, HS_ERR_BOUNDS);
                return 0.f;
            }
        }
        return __ldg(tt.fop32 + (long long)(rho + zr) * tt.ld + b);
    };

    // ---- slow pass (defined here, run below): exact per-level test -----------
    // scan(z, write, slot, dry): level sums of row z in Eq. 2 order; returns
    // the hit mask over levels and, when write is set, appends the records
    // from slot.  A dry run reads no FP32 copy.
    auto scan = [&](int z, bool write, uint32_t rslot, bool dry) -> uint32_t {
        float acc = 0.f, ab = 0.f;
        uint32_t hits = 0u;
        float thr[H];
        static_for<0, H>([&](auto M) { thr[M] = thr_of(M, z); });
        // The decision of Section III: HP_k(z, f) > TA(k, z), HP_k formed in
        // the order of Eq. 2 (ascending m) in FP32.  The pass is rare, so
        // what it costs is its code run cold from the instruction cache; the
        // FP32 form compiles nothing else.
        if constexpr (C::ES == 4) {
            // FP32 storage: the stored values' chain decides
            static_for<0, H>([&](auto M) {
                constexpr int m = M + 1;
                const int rho = z >= 0 ? z / m : -((-z) / m);
                const float v = sld(M, bidx[M] + rho * C::W(m));
                acc = (m == 1) ? v : acc + v;
                if (acc > thr[M]) {
                    hits |= 1u << M;
                    if (write)
                        put_record(tt.rec, rslot++, tt.cap, (uint32_t)f, z, m, 0u, acc);
                }
            });
        } else {
            // 16-bit storage.  With the FP32 copy: a level whose 16-bit sum
            // lies within the storage error of its threshold is decided by the
            // copy's chain (the same FP32 numbers the FP32 path forms), all of
            // whose H values are loaded at once; without it the 16-bit sum
            // decides and the record is flagged.
            float pw[H];
            uint32_t need = 0u, nearm = 0u;
            static_for<0, H>([&](auto M) {
                constexpr int m = M + 1;
                const int rho = z >= 0 ? z / m : -((-z) / m);
                const float v = sld(M, bidx[M] + rho * C::W(m));
                acc = (m == 1) ? v : acc + v;
                ab += fabsf(v);
                pw[M] = acc;
                const float band = p.delta * ab + p.band_abs;
                if (tt.fop32 != nullptr) {
                    if (!(acc == acc && acc + band < thr[M]))
                        need |= 1u << M;
                } else {
                    hits |= (acc > thr[M] ? 1u : 0u) << M;
                    nearm |= (fabsf(acc - thr[M]) <= band ? 1u : 0u) << M;
                }
            });
            if (need != 0u && !dry) {
                float w[H];
                static_for<0, H>([&](auto M) {
                    constexpr int m = M + 1;
                    const int rho = z >= 0 ? z / m : -((-z) / m);
                    w[M] = copy_at(rho, f / m);
                });
                float c = 0.f;
                static_for<0, H>([&](auto M) {
                    constexpr int m = M + 1;
                    c = (m == 1) ? w[M] : c + w[M];
                    if (((need >> M) & 1u) && c > thr[M]) {
                        hits |= 1u << M;
                        pw[M] = c;
                    }
                });
            }
            if (write) {
                const uint32_t fl = tt.fop32 != nullptr ? 0u : HS_FLAG_LOWP;
                static_for<0, H>([&](auto M) {
                    if ((hits >> M) & 1u)
                        put_record(tt.rec, rslot++, tt.cap, (uint32_t)f, z, M + 1,
                                   fl | (((nearm >> M) & 1u) ? HS_FLAG_NEAR : 0u), pw[M]);
                });
            }
        }
        return hits;
    };

    // FP32: the level sums of row z (Eq. 2 order) into pw, the hit mask out
    auto scan32 = [&](int z, float (&pw)[H]) -> uint32_t {
        float acc = 0.f;
        uint32_t hits = 0u;
        float thr[H];
        static_for<0, H>([&](auto M) { thr[M] = thr_of(M, z); });
        static_for<0, H>([&](auto M) {
            constexpr int m = M + 1;
            const int rho = z >= 0 ? z / m : -((-z) / m);
            acc = (m == 1) ? sld(M, bidx[M] + rho * C::W(m))
                           : acc + sld(M, bidx[M] + rho * C::W(m));
            pw[M] = acc;
            hits |= (acc > thr[M] ? 1u : 0u) << M;
        });
        return hits;
    };

    // A dry run of the exact pass on this thread's centre row while the
    // copies are in flight (the values read are discarded): the pass's code
    // is then in the instruction cache when a marked pair needs it.  On
    // 16-bit planes the dry run reads no FP32 copy.
    if constexpr (C::ES == 4) {
        float pw[H];
        const uint32_t dry = scan32(0, pw);
        asm volatile("" ::"r"(dry), "f"(pw[H - 1]));
    } else if (tt.pend == nullptr) {
        const uint32_t dry = scan(0, false, 0u, true);
        asm volatile("" ::"r"(dry));
    }

    // CTA-uniform outcome of the bounded wait for the stage
    const bool ok = !any_of(!mbar_wait_bounded(bar, parity, kWaitLimitNs));

    // ---- fast pass: every row pair, group prefilter ------------------------------
    // d_g = HP_b - bound_g (b the last level of group g) has its sign bit set
    // exactly when HP_b < bound_g (IEEE addition is sign-exact without
    // flush-to-zero), so AND-ing the sign bits of every group's d leaves bit
    // 31 set iff no group of the pair can hold a hit.  The bounds ride along
    // in the sums: the last level of group g (the one reloaded least often)
    // carries c_g = bound_{g-1} - bound_g (c_0 = -bound_0) from the moment it
    // is loaded, so the running sum over the groups is d_g itself and no
    // separate subtraction is needed.  The host lowers the bounds by the
    // rounding this mixing of signs adds.
    float2 cg[C::G];
    static_for<0, C::G>([&](auto g) {
        const float c = g == 0 ? -p.tmin[0] : p.tmin[g - 1] - p.tmin[g];
        cg[g] = make_float2(c, c);
    });
    // the group whose last level is m, or -1
    auto carrier_of = [](int m) {
        for (int g = 0; g < C::G; ++g)
            if (C::GHI(g) == m)
                return g;
        return -1;
    };
    uint32_t negbits = 0u;
    uint64_t mask = 0ull;
    // Each pair's sign AND is shifted into clear[w] (one funnel shift per
    // pair; set = no group can hit; pairs 0..31 in word 0, the rest in word
    // 1) and turned into the mask once at the end.
    uint32_t clear[2] = {0u, 0u};
    float2 cur[H];
    // Each group's tree sum, and the sums of its two halves, are kept from
    // pair to pair and recomputed only at the pairs where one of their levels
    // was reloaded (m divides zz), so the values are exactly those of a full
    // recomputation of the tree.
    float2 gsum[C::G], ghalf[C::G][2];
    auto pair_test = [&](auto ZZ) -> uint32_t {
        constexpr int zz = decltype(ZZ)::value;
        float2 acc = make_float2(0.f, 0.f);
        uint32_t sgn = 0xffffffffu;
        static_for<0, C::G>([&](auto g) {
            constexpr int lo = C::GLO(g), hi = C::GHI(g), mid = (lo + hi) / 2;
            if constexpr (lo == hi) {
                if constexpr (zz == 0 || reloads_any(zz, lo, hi))
                    gsum[g] = cur[lo - 1];
            } else {
                constexpr bool cl = zz == 0 || reloads_any(zz, lo, mid);
                constexpr bool cr = zz == 0 || reloads_any(zz, mid + 1, hi);
                if constexpr (cl)
                    ghalf[g][0] = tree_sum<lo - 1, mid - 1>(cur);
                if constexpr (cr)
                    ghalf[g][1] = tree_sum<mid, hi - 1>(cur);
                if constexpr (cl || cr)
                    gsum[g] = __fadd2_rn(ghalf[g][0], ghalf[g][1]);
            }
            if constexpr (g == 0)
                acc = gsum[g];
            else
                acc = __fadd2_rn(acc, gsum[g]);
            sgn &= __float_as_uint(acc.x) & __float_as_uint(acc.y);
        });
        return sgn; // bit 31 clear: the pair may hold a hit
    };
    auto record = [&](auto ZZ, uint32_t sgn) {
        constexpr int w = decltype(ZZ)::value < 32 ? 0 : 1;
        clear[w] = __funnelshift_l(sgn, clear[w], 1); // (clear << 1) | sgn >> 31
    };
    // the value of level m at the pair (tv, bv), with its group's bound share
    auto put = [&](auto M, float tv, float bv) {
        constexpr int g = carrier_of(decltype(M)::value + 1);
        if constexpr (g >= 0)
            cur[M] = __fadd2_rn(make_float2(tv, bv), cg[g]);
        else
            cur[M] = make_float2(tv, bv);
    };
    bool out_ok = true;
    if (ok) {
        // template z = 0: every stretch reads the centre row
        static_for<0, H>([&](auto M) {
            const float v = sld(M, bidx[M]);
            put(M, v, v);
            if constexpr (SIGNCHK)
                negbits |= __float_as_uint(v);
        });
        record(std::integral_constant<int, 0>{}, pair_test(std::integral_constant<int, 0>{}));
        // pairs (+zz, -zz): reload the value of m only when m divides zz
        static_for<1, Z + 1>([&](auto ZZ) {
            constexpr int zz = ZZ;
            if constexpr (RT) {
                if (zz > zr) { // past the plane's rows: nothing to mark
                    record(ZZ, 0xffffffffu);
                    return;
                }
            }
            if constexpr (BANDED && zz == C::RB + 1) {
                // the outer rows: a wait bounded in time and in tries, inline
                // (a call inside the unrolled walk would spill it); the asm's
                // memory clobber keeps the loads below it
                bool got = mbar_try_wait_hint(bar_out, parity, 1000000u);
                if (!got) {
                    const uint64_t t0 = globaltimer_ns();
                    for (uint32_t it = 0; !got && it < kBandWaitTries; ++it) {
                        got = mbar_try_wait_hint(bar_out, parity, 1000000u);
                        if (!got && globaltimer_ns() - t0 > kWaitLimitNs)
                            break;
                    }
                }
                out_ok = got;
            }
            static_for<0, H>([&](auto M) {
                constexpr int m = M + 1;
                if constexpr (zz % m == 0) {
                    constexpr int off = (zz / m) * C::W(m);
                    const float tv = sld(M, bidx[M] + off);
                    const float bv = sld(M, bidx[M] - off);
                    put(M, tv, bv);
                    if constexpr (SIGNCHK)
                        negbits |= __float_as_uint(tv) | __float_as_uint(bv);
                }
            });
            record(ZZ, pair_test(ZZ));
        });
        // word 0 holds pairs 0 .. n0-1 with pair zz at bit n0-1-zz, word 1
        // pairs 32 .. Z with pair zz at bit Z-zz; reverse the bits into the
        // mask (bit zz = the pair may hold a hit)
        static_assert(Z <= 63, "two mask words");
        constexpr int n0 = Z + 1 < 32 ? Z + 1 : 32;
        mask = (uint64_t)(__brev(~clear[0]) >> (32 - n0));
        if constexpr (Z >= 32)
            mask |= (uint64_t)((__brev(~clear[1]) >> (63 - Z)) &
                               (uint32_t)((1ull << (Z - 31)) - 1ull)) << 32;
        if constexpr (BANDED)
            out_ok = !any_of(!out_ok); // CTA-uniform, like ok
    }
    if (!ok || !out_ok) {
        if (tid == 0)
            set_status(tt.counters, HS_ERR_TIMEOUT);
        mbar_wait_bounded(bar, parity, kWaitLimitNs); // let copies in flight land
        if constexpr (BANDED)
            mbar_wait_bounded(bar_out, parity, kWaitLimitNs);
        return false;
    }
    if (!valid)
        mask = 0ull;
    else if (negbits >> 31)
        mask = (zr == 63) ? ~0ull : ((1ull << (zr + 1)) - 1ull);

    while (__any_sync(0xffffffffu, mask != 0ull)) {
        int zz = -1;
        if (mask != 0ull) {
            zz = __ffsll((long long)mask) - 1;
            mask &= mask - 1ull;
        }
        uint32_t ht = 0u, hb = 0u;
        if constexpr (C::ES == 4) {
            // both rows' sums stay in registers for the write
            float pt[H], pb[H];
            if (zz >= 0) {
                ht = scan32(zz, pt);
                if (zz > 0)
                    hb = scan32(-zz, pb);
            }
            uint32_t rsl = warp_reserve(tt.counters, (uint32_t)(__popc(ht) + __popc(hb)));
            static_for<0, H>([&](auto M) {
                if ((ht >> M) & 1u)
                    put_record(tt.rec, rsl++, tt.cap, (uint32_t)f, zz, M + 1, 0u, pt[M]);
            });
            static_for<0, H>([&](auto M) {
                if ((hb >> M) & 1u)
                    put_record(tt.rec, rsl++, tt.cap, (uint32_t)f, -zz, M + 1, 0u, pb[M]);
            });
        } else {
            if (tt.pend != nullptr) {
                // deferred: the marked pair goes to the pending list and the
                // recheck kernel decides both rows from the FP32 copy (all
                // pairs' reads in flight together, after this grid); only a
                // pair the full list cannot take is decided here
                const uint32_t ps = warp_reserve(tt.pend_count, zz >= 0 ? 1u : 0u);
                if (zz >= 0 && ps < tt.pend_cap) {
                    tt.pend[ps] = make_uint2((uint32_t)f, (uint32_t)zz);
                    zz = -1;
                }
                if (!__any_sync(0xffffffffu, zz >= 0))
                    continue;
            }
            if (zz >= 0) {
                ht = scan(zz, false, 0u, false);
                if (zz > 0)
                    hb = scan(-zz, false, 0u, false);
            }
            uint32_t rsl = warp_reserve(tt.counters, (uint32_t)(__popc(ht) + __popc(hb)));
            if (ht)
                scan(zz, true, rsl, false);
            if (hb)
                scan(-zz, true, rsl + (uint32_t)__popc(ht), false);
        }
    }
    return true;
}

// Resident CTAs the register budget is sized for: as many as shared memory
// allows while each thread keeps 128 registers (the fast pass holds 16
// packed row-pair values, 16 span indices and the group bounds).
template <int NT, int H, int TB, typename T>
constexpr int resident_ctas()
{
    return cmin(Cfg<NT, H, TB, T>::CTAS_SMEM, 65536 / (TB * 128));
}

// One plane.  Grid-stride over the tile order: with one CTA per tile each CTA
// sums one tile; with a smaller grid the CTAs stay resident and walk several
// tiles, saving the launch and teardown of a CTA per tile.
template <int NT, int H, int TB, typename T, bool SIGNCHK = true, bool BANDED = false,
          bool RT = false>
__global__ void __launch_bounds__(TB, (resident_ctas<NT, H, TB, T>()))
    staged_kernel(const __grid_constant__ Params<NT, H, T> p)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_storage[2];
    const uint32_t sbase = smem_addr(smem);
    const uint32_t bar = smem_addr(&bar_storage[0]);
    const uint32_t bar_out = smem_addr(&bar_storage[1]);
    if (threadIdx.x == 0) {
        static_for<0, H>([&](auto M) { prefetch_tmap(&p.maps[M]); });
        mbar_init(bar, 1);
        if constexpr (BANDED) {
            prefetch_tmap(&p.split1[0]);
            prefetch_tmap(&p.split1[1]);
            mbar_init(bar_out, 1);
        }
    }
    __syncthreads();
    const TileTarget tt{p.maps,     p.split1,   p.fop32, p.n,
                        p.ld,       p.rec,      p.counters, p.cap,
                        (p.nt_rt - 1) / 2, p.nt_rt, p.pend,  p.pend_count,
                        p.pend_cap};
    uint32_t parity = 0;
    for (int i = (int)blockIdx.x; i < p.n_slots; i += (int)gridDim.x, parity ^= 1u) {
        const int slot = p.tile_lo + i;
        const int f0 = (p.order ? (int)__ldg(p.order + slot) : slot) * TB;
        if (threadIdx.x == 0) {
            if constexpr (BANDED)
                issue_tile_banded<NT, H, TB, T>(tt, f0, sbase, bar, bar_out);
            else
                issue_tile<NT, H, TB, T, RT>(tt, f0, sbase, bar);
        }
        if (!sum_tile<NT, H, TB, T, Params<NT, H, T>, CtaOr, SIGNCHK, BANDED, RT>(
                p, tt, f0, smem, bar, parity, CtaOr{}, bar_out))
            break;
        __syncthreads(); // the stage is free before the next tile's boxes land
    }
}

// One plane, pipelined and warp-specialised: one persistent CTA per SM with
// an S-stage ring of tile stages.  A producer warp issues each tile's boxes
// as soon as its stage is released; NC consumer groups of TB threads sum the
// tiles (group c takes iterations c, c + NC, ...), so the copies of the next
// tiles are in flight while the groups sum.  full[s] completes once per use
// of stage s (the boxes landed), empty[s] once per release.  Iteration j uses
// stage j % S in its phase k = j / S.  Before waiting on full[s] for phase k a
// consumer waits on empty[s] for phase k - 1, so a parity it waits for is
// never that of a phase two behind (2 S is a multiple of NC: iteration j - 2S
// belongs to the same group, which released it already).
template <int NT, int H, int TB, int NC, int S, typename T>
__global__ void __launch_bounds__(NC *TB + 32, 1)
    pipe_kernel(const __grid_constant__ Params<NT, H, T> p)
{
    static_assert((2 * S) % NC == 0 && S >= 2 && NC >= 1, "ring shape");
    using C = Cfg<NT, H, TB, T>;
    constexpr int STAGE = round_up(C::SMEM, 1024);
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full_bar[S], empty_bar[S];
    __shared__ int issued; // iterations the producer issued
    const uint32_t sbase = smem_addr(smem);
    const TileTarget tt{p.maps, nullptr,  p.fop32, p.n,          p.ld,
                        p.rec,  p.counters, p.cap, (NT - 1) / 2, NT};
    const int G = (int)gridDim.x;
    const int n_it = (int)blockIdx.x < p.n_slots ? (p.n_slots - 1 - (int)blockIdx.x) / G + 1 : 0;
    auto tile_f0 = [&](int j) {
        const int slot = p.tile_lo + (int)blockIdx.x + j * G;
        return (p.order ? (int)__ldg(p.order + slot) : slot) * TB;
    };
    if (threadIdx.x == 0) {
        static_for<0, H>([&](auto M) { prefetch_tmap(&p.maps[M]); });
        static_for<0, S>([&](auto st) {
            mbar_init(smem_addr(&full_bar[st]), 1);
            mbar_init(smem_addr(&empty_bar[st]), 1);
        });
        issued = 0;
    }
    __syncthreads();
    const int group = (int)threadIdx.x / TB;
    if (group == NC) { // producer warp
        if ((threadIdx.x & 31u) == 0u) {
            for (int j = 0; j < n_it; ++j) {
                const int st = j % S, k = j / S;
                if (k >= 1 && !mbar_wait_bounded(smem_addr(&empty_bar[st]), (uint32_t)(k - 1) & 1u,
                                                 kWaitLimitNs)) {
                    set_status(p.counters, HS_ERR_TIMEOUT);
                    break;
                }
                issue_tile<NT, H, TB, T>(tt, tile_f0(j), sbase + st * STAGE,
                                         smem_addr(&full_bar[st]));
                *(volatile int *)&issued = j + 1;
            }
        }
        __syncwarp();
    } else { // consumer group
        const int gid = 1 + group;
        auto any_of = [gid](bool v) { return group_or(gid, TB, v); };
        for (int j = group; j < n_it; j += NC) {
            const int st = j % S, k = j / S;
            const uint32_t full = smem_addr(&full_bar[st]), empty = smem_addr(&empty_bar[st]);
            if (k >= 1 && any_of(!mbar_wait_bounded(empty, (uint32_t)(k - 1) & 1u, kWaitLimitNs))) {
                if (threadIdx.x % TB == 0)
                    set_status(p.counters, HS_ERR_TIMEOUT);
                break;
            }
            if (!sum_tile<NT, H, TB, T>(p, tt, tile_f0(j), smem + st * STAGE, full,
                                        (uint32_t)k & 1u, any_of))
                break;
            group_sync(gid, TB); // the group is done with stage st
            if (threadIdx.x % TB == 0)
                mbar_arrive(empty);
        }
    }
    __syncthreads();
    // after a timeout, let every issued copy land before the CTA exits
    if (threadIdx.x == 0) {
        const int n_issued = *(volatile int *)&issued;
        for (int st = 0; st < S; ++st) {
            int last = -1;
            for (int j = st; j < n_issued; j += S)
                last = j;
            if (last >= 0)
                mbar_wait_bounded(smem_addr(&full_bar[st]), (uint32_t)(last / S) & 1u,
                                  kWaitLimitNs);
        }
    }
}

// One beam of a batched launch, carried in the kernel parameters: its
// descriptors, size, output, and the end of its tiles in the launch's slots.
template <int H>
struct BeamParam {
    CUtensorMap maps[H];
    CUtensorMap split1[2]; // level 1 in row bands (centre, outer side)
    const float *fop32;
    long long n;
    long long ld;
    hs_cand *rec;
    uint32_t *counters;
    uint32_t cap;
    int tile_end; // one past the beam's last slot (cumulative over the launch)
};

// Largest kernel parameter block the launch accepts.
constexpr int kParamBytes = 32764;

template <int NT, int H, typename T>
struct BatchParams {
    // beams per launch: as many as the parameter block holds (at most 32)
    static constexpr int K =
        cmin(32, (kParamBytes - 128) / (int)sizeof(BeamParam<H>));
    float tmin[n_groups(H)];
    const float *ta;
    const uint32_t *order; // per-beam tile order of the whole batch (device) or null
    float delta;
    float band_abs;
    int n_beams;           // beams of this launch
    int slot_base;         // first slot of this launch in the batch's order table
    int n_slots;           // tiles of this launch
    BeamParam<H> beam[K];
};

// Many beams in one launch.  The descriptors of every beam sit in the
// parameter block (constant bank), like those of a single-plane launch, so a
// tile's copies need no proxy fence on descriptors in global memory; the CTAs
// walk the concatenated tiles of the launch's beams grid-stride (one tile per
// CTA when the grid covers them) and find each tile's beam by a CTA-uniform
// scan of the cumulative tile ends.
template <int NT, int H, int TB, typename T, bool SIGNCHK = true, bool BANDED = false>
__global__ void __launch_bounds__(TB, (resident_ctas<NT, H, TB, T>()))
    batched_kernel(const __grid_constant__ BatchParams<NT, H, T> p)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_storage[2];
    const uint32_t sbase = smem_addr(smem);
    const uint32_t bar = smem_addr(&bar_storage[0]);
    const uint32_t bar_out = smem_addr(&bar_storage[1]);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        if constexpr (BANDED)
            mbar_init(bar_out, 1);
    }
    __syncthreads();
    int cur = -1; // beam whose descriptors thread 0 last prefetched
    uint32_t parity = 0;
    for (int i = (int)blockIdx.x; i < p.n_slots; i += (int)gridDim.x, parity ^= 1u) {
        int b = 0;
        while (b + 1 < p.n_beams && i >= p.beam[b].tile_end)
            ++b;
        const BeamParam<H> &bp = p.beam[b];
        const int local = i - (b ? p.beam[b - 1].tile_end : 0);
        const int tile = p.order ? (int)__ldg(p.order + p.slot_base + i) : local;
        const TileTarget tt{bp.maps,     bp.split1, bp.fop32,     bp.n, bp.ld,
                            bp.rec,      bp.counters, bp.cap, (NT - 1) / 2, NT};
        if (threadIdx.x == 0) {
            if (b != cur) {
                static_for<0, H>([&](auto M) { prefetch_tmap(&bp.maps[M]); });
                if constexpr (BANDED) {
                    prefetch_tmap(&bp.split1[0]);
                    prefetch_tmap(&bp.split1[1]);
                }
            }
            if constexpr (BANDED)
                issue_tile_banded<NT, H, TB, T>(tt, tile * TB, sbase, bar, bar_out);
            else
                issue_tile<NT, H, TB, T>(tt, tile * TB, sbase, bar);
        }
        cur = b;
        if (!sum_tile<NT, H, TB, T, BatchParams<NT, H, T>, CtaOr, SIGNCHK, BANDED>(
                p, tt, tile * TB, smem, bar, parity, CtaOr{}, bar_out))
            break;
        __syncthreads();
    }
}

// Packed batch: every beam lies in one plane [NT][ld], side by side along the
// bins (beam b at bins [off_b, off_b + n_b) of every row), so one set of
// descriptors addresses them all and one launch sums every tile of every beam.
template <int NT, int H, typename T>
struct PackedParams {
    CUtensorMap maps[H];    // spans of the packed plane, one box per stretch factor
    CUtensorMap split1[2];  // level 1 in row bands
    float tmin[n_groups(H)];
    const float *ta;
    const float *fop32;     // FP32 copy of the packed plane (same layout), or null
    const uint2 *tiles;     // per slot: (beam, tile of that beam), in run order
    const PackedBeam *beams;
    long long ld;           // row pitch of the packed plane (elements)
    float delta;
    float band_abs;
    int n_slots;
};

template <int NT, int H, int TB, typename T, bool SIGNCHK = true, bool BANDED = false>
__global__ void __launch_bounds__(TB, (resident_ctas<NT, H, TB, T>()))
    packed_kernel(const __grid_constant__ PackedParams<NT, H, T> p)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_storage[2];
    const uint32_t sbase = smem_addr(smem);
    const uint32_t bar = smem_addr(&bar_storage[0]);
    const uint32_t bar_out = smem_addr(&bar_storage[1]);
    if (threadIdx.x == 0) {
        static_for<0, H>([&](auto M) { prefetch_tmap(&p.maps[M]); });
        mbar_init(bar, 1);
        if constexpr (BANDED) {
            prefetch_tmap(&p.split1[0]);
            prefetch_tmap(&p.split1[1]);
            mbar_init(bar_out, 1);
        }
    }
    __syncthreads();
    uint32_t parity = 0;
    for (int i = (int)blockIdx.x; i < p.n_slots; i += (int)gridDim.x, parity ^= 1u) {
        const uint2 e = __ldg(p.tiles + i);
        const PackedBeam &pb = p.beams[e.x];
        const long long off = __ldg(&pb.off);
        const TileTarget tt{p.maps,
                            p.split1,
                            p.fop32 ? p.fop32 + off : nullptr,
                            __ldg(&pb.n),
                            p.ld,
                            (hs_cand *)__ldg((const unsigned long long *)&pb.rec),
                            (uint32_t *)__ldg((const unsigned long long *)&pb.counters),
                            __ldg(&pb.cap),
                            (NT - 1) / 2,
                            NT};
        const int f0 = (int)e.y * TB;
        if (threadIdx.x == 0) {
            if constexpr (BANDED)
                issue_tile_banded<NT, H, TB, T>(tt, f0, sbase, bar, bar_out, (int)off);
            else
                issue_tile<NT, H, TB, T>(tt, f0, sbase, bar, (int)off);
        }
        if (!sum_tile<NT, H, TB, T, PackedParams<NT, H, T>, CtaOr, SIGNCHK, BANDED>(
                p, tt, f0, smem, bar, parity, CtaOr{}, bar_out))
            break;
        __syncthreads();
    }
}

// Zero the counter pair of every beam of a packed batch.
__global__ void reset_packed(const PackedBeam *beams, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        beams[i].counters[0] = 0u;
        beams[i].counters[1] = 0u;
    }
}

template <int NT, int H, int TB, typename T, bool SIGNCHK = true, bool BANDED = false>
cudaError_t launch_packed_one(const PackedBatch &a, cudaStream_t s)
{
    using C = Cfg<NT, H, TB, T>;
    PackedParams<NT, H, T> p;
    std::memset(&p, 0, sizeof p);
    std::memcpy(p.maps, a.maps, sizeof(CUtensorMap) * H);
    std::memcpy(p.split1, a.split1, sizeof(CUtensorMap) * 2);
    for (int g = 0; g < C::G; ++g)
        p.tmin[g] = a.tmin_host[g];
    p.ta = a.ta;
    p.fop32 = a.fop32;
    p.tiles = a.tiles;
    p.beams = a.beams;
    p.ld = a.ld;
    p.delta = a.delta;
    p.band_abs = a.band_abs;
    p.n_slots = a.n_tiles;
    if (a.n_beams > 0) {
        reset_packed<<<(a.n_beams + 127) / 128, 128, 0, s>>>(a.beams, a.n_beams);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    if (p.n_slots <= 0)
        return cudaSuccess;
    auto kern = packed_kernel<NT, H, TB, T, SIGNCHK, BANDED>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess)
        return e;
    int grid = p.n_slots;
    if (a.grid_per_sm > 0 && a.sms * a.grid_per_sm < grid)
        grid = a.sms * a.grid_per_sm;
    kern<<<grid, TB, C::SMEM, s>>>(p);
    return cudaGetLastError();
}

// Counter pairs to clear before a batched launch, in the parameter block.
struct CounterList {
    static constexpr int K = 1024;
    uint32_t *c[K];
    int n;
};

__global__ void reset_counter_list(const __grid_constant__ CounterList l)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < l.n) {
        l.c[i][0] = 0u;
        l.c[i][1] = 0u;
    }
}

template <int NT, int H, int TB, typename T, bool SIGNCHK = true, bool BANDED = false,
          bool RT = false>
cudaError_t launch_one(const StagedLaunch &a, cudaStream_t s)
{
    using C = Cfg<NT, H, TB, T>;
    Params<NT, H, T> p;
    std::memset(&p, 0, sizeof p);
    std::memcpy(p.maps, a.maps, sizeof(CUtensorMap) * H);
    if constexpr (BANDED)
        std::memcpy(p.split1, a.split1, sizeof(CUtensorMap) * 2);
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
    p.ld = a.ld;
    p.tile_lo = a.tile_lo;
    p.n_slots = a.tile_hi - a.tile_lo;
    p.nt_rt = a.nt_rt > 0 ? a.nt_rt : NT;
    if constexpr (sizeof(T) == 2) {
        if (a.fop32 != nullptr) {
            p.pend = a.pend;
            p.pend_count = a.pend_count;
            p.pend_cap = a.pend_cap;
        }
    }
    if (p.n_slots <= 0)
        return cudaSuccess;
    if (p.nt_rt > NT || p.nt_rt % 2 == 0 || (!RT && p.nt_rt != NT))
        return cudaErrorInvalidValue;
    auto kern = staged_kernel<NT, H, TB, T, SIGNCHK, BANDED, RT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e == cudaSuccess) // all of the unified L1/shared storage as shared memory
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess)
        return e;
    int grid = p.n_slots;
    if (a.grid_per_sm > 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess)
            return e;
        grid = sms * a.grid_per_sm < grid ? sms * a.grid_per_sm : grid;
    }
    kern<<<grid, TB, C::SMEM, s>>>(p);
    return cudaGetLastError();
}

// A plane declared non-negative, one CTA per tile.  FP32 planes load level 1
// in row bands (169 against 173 us on the 85 x 2^21 plane); 16-bit planes
// keep one barrier (the banded form measured 2 us slower there).
template <int NT, int H, int TB, typename T>
cudaError_t launch_nonneg(const StagedLaunch &a, cudaStream_t s)
{
    if constexpr (sizeof(T) == 4) {
        if (a.split1)
            return launch_one<NT, H, TB, T, false, true>(a, s);
    }
    return launch_one<NT, H, TB, T, false>(a, s);
}

template <int NT, int H, int TB, int NC, int S, typename T>
cudaError_t launch_pipe(const StagedLaunch &a, cudaStream_t s)
{
    using C = Cfg<NT, H, TB, T>;
    constexpr int SMEM = S * round_up(C::SMEM, 1024);
    static_assert(SMEM <= 232448 - 2048, "ring stages exceed the shared memory of a CTA");
    Params<NT, H, T> p;
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
    p.ld = a.ld;
    p.tile_lo = a.tile_lo;
    p.n_slots = a.tile_hi - a.tile_lo;
    if (p.n_slots <= 0)
        return cudaSuccess;
    auto kern = pipe_kernel<NT, H, TB, NC, S, T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess)
        return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    const int grid = sms < p.n_slots ? sms : p.n_slots;
    kern<<<grid, NC * TB + 32, SMEM, s>>>(p);
    return cudaGetLastError();
}

template <int NT, int H, int TB, typename T, bool SIGNCHK = true, bool BANDED = false>
cudaError_t launch_batch_one(const StagedBatch &a, cudaStream_t s)
{
    using C = Cfg<NT, H, TB, T>;
    using BP = BatchParams<NT, H, T>;
    static_assert(sizeof(BP) <= kParamBytes, "parameter block");
    cudaError_t e = cudaSuccess;
    for (int b0 = 0; b0 < a.n_beams && e == cudaSuccess; b0 += CounterList::K) {
        CounterList l;
        l.n = std::min(CounterList::K, a.n_beams - b0);
        for (int i = 0; i < l.n; ++i)
            l.c[i] = a.beams[b0 + i].counters;
        reset_counter_list<<<(l.n + 127) / 128, 128, 0, s>>>(l);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return e;
    auto kern = batched_kernel<NT, H, TB, T, SIGNCHK, BANDED>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess)
        return e;
    BP p; // the parameter block, copied into the launch
    int slot = 0;
    for (int b0 = 0; b0 < a.n_beams; b0 += BP::K) {
        std::memset(&p, 0, sizeof p);
        for (int g = 0; g < C::G; ++g)
            p.tmin[g] = a.tmin_host[g];
        p.ta = a.ta;
        p.order = a.order;
        p.delta = a.delta;
        p.band_abs = a.band_abs;
        p.n_beams = std::min(BP::K, a.n_beams - b0);
        p.slot_base = slot;
        int end = 0;
        for (int j = 0; j < p.n_beams; ++j) {
            const StagedBatchBeam &src = a.beams[b0 + j];
            BeamParam<H> &d = p.beam[j];
            std::memcpy(d.maps, src.maps, sizeof(CUtensorMap) * H);
            std::memcpy(d.split1, src.split1, sizeof(CUtensorMap) * 2);
            d.fop32 = src.fop32;
            d.n = src.n;
            d.ld = src.ld;
            d.rec = src.rec;
            d.counters = src.counters;
            d.cap = src.cap;
            end += src.tiles;
            d.tile_end = end;
        }
        p.n_slots = end;
        slot += end;
        if (end == 0)
            continue;
        int grid = end;
        if (a.grid_per_sm > 0 && a.sms * a.grid_per_sm < grid)
            grid = a.sms * a.grid_per_sm;
        kern<<<grid, TB, C::SMEM, s>>>(p);
        e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

template <int NT, int H, int TB, typename T>
void box_of(int m, int *w, int *rows)
{
    *w = Cfg<NT, H, TB, T>::W(m);
    *rows = Cfg<NT, H, TB, T>::ROWS(m);
}


// ---- entry points of one shape, for the registry in hs_staged.cu -----------------

template <int NT, int H, int TB, typename T>
cudaError_t plane_checked(const StagedLaunch &a, cudaStream_t s)
{
    return launch_one<NT, H, TB, T>(a, s);
}

template <int NT, int H, int TB, typename T>
cudaError_t plane_nonneg(const StagedLaunch &a, cudaStream_t s)
{
    return launch_nonneg<NT, H, TB, T>(a, s);
}

template <int NT, int H, int TB, int NC, int S, typename T>
cudaError_t plane_ring(const StagedLaunch &a, cudaStream_t s)
{
    return launch_pipe<NT, H, TB, NC, S, T>(a, s);
}

template <int NT, int H, int TB, typename T>
cudaError_t batch_fn(const StagedBatch &a, cudaStream_t s)
{
    return a.assume_nonneg ? launch_batch_one<NT, H, TB, T, false, sizeof(T) == 4>(a, s)
                           : launch_batch_one<NT, H, TB, T>(a, s);
}

template <int NT, int H, int TB, typename T>
cudaError_t packed_fn(const PackedBatch &a, cudaStream_t s)
{
    return a.assume_nonneg ? launch_packed_one<NT, H, TB, T, false, sizeof(T) == 4>(a, s)
                           : launch_packed_one<NT, H, TB, T>(a, s);
}

// A plane shape: the sign-checked kernel (every launch form) and, when
// NONNEG, the kernel for planes declared non-negative.
template <int NT, int H, int TB, typename T, int DT, bool NONNEG>
ShapeEntry plane_entry()
{
    return ShapeEntry{StagedShape{NT, H, TB, DT}, Cfg<NT, H, TB, T>::SMEM, &box_of<NT, H, TB, T>,
                      &plane_checked<NT, H, TB, T>,
                      NONNEG ? &plane_nonneg<NT, H, TB, T> : nullptr, false};
}

template <int NT, int H, int TB, typename T>
cudaError_t plane_checked_rt(const StagedLaunch &a, cudaStream_t s)
{
    return launch_one<NT, H, TB, T, true, false, true>(a, s);
}

template <int NT, int H, int TB, typename T>
cudaError_t plane_nonneg_rt(const StagedLaunch &a, cudaStream_t s)
{
    return launch_one<NT, H, TB, T, false, false, true>(a, s);
}

// A family with runtime rows: serves every odd template count up to NT at
// H levels (one barrier; sign-checked and declared non-negative).
template <int NT, int H, int TB, typename T, int DT>
ShapeEntry plane_entry_rt()
{
    return ShapeEntry{StagedShape{NT, H, TB, DT}, Cfg<NT, H, TB, T>::SMEM, &box_of<NT, H, TB, T>,
                      &plane_checked_rt<NT, H, TB, T>, &plane_nonneg_rt<NT, H, TB, T>, true};
}

template <int NT, int H, int TB, typename T, int DT>
BatchEntry batch_entry()
{
    return BatchEntry{StagedShape{NT, H, TB, DT}, BatchParams<NT, H, T>::K, &batch_fn<NT, H, TB, T>,
                      &packed_fn<NT, H, TB, T>};
}

template <int NT, int H, int TB, int NC, int S, typename T, int DT>
RingEntry ring_entry()
{
    return RingEntry{StagedShape{NT, H, TB, DT}, NC, S, &plane_ring<NT, H, TB, NC, S, T>};
}

} // namespace
} // namespace hs
