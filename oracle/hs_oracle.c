/*
 * hs_oracle.c -- plain FP64 CPU reference ("oracle") for the harmonic-summing
 * stage of Fourier-domain acceleration search (Wang, Thiagaraj & Sinnen,
 * "Harmonic-summing Module of SKA on FPGA", arXiv 1805.12258).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file.  It shares no code, header,
 * table or helper with the CUDA library; the two meet only through the seeded
 * inputs that the tests hand to both.
 *
 * What it computes (Section III of the paper):
 *   - the filter-output plane (FOP) has N_temp rows (templates) indexed by a
 *     signed i in [-(N_temp-1)/2, (N_temp-1)/2] and N_chan columns (bins) j;
 *   - Eq. 1, stretch plane:   SP_k(i,j) = FOP(rho(i,k), floor(j/k));
 *   - Eq. 2, harmonic plane:  HP_1 = FOP,  HP_k = HP_{k-1} + SP_k;
 *   - detection: a point of HP_k is a candidate when it exceeds the threshold
 *     TA(k,i) of its level and row (strict '>': the paper does not say which
 *     comparison; strict is the reading taken).
 * rho() is the row rounding.  The paper writes floor(i/k) and says the two
 * template groups (i>0, i<0) are stretched separately; the default reading
 * mirrors the groups, rho(i,k) = sign(i)*floor(|i|/k) ("symmetric"); the
 * literal floor toward -infinity is the alternative ("floor").
 *
 * A second index map ("harmonic fraction") sums, for level k, the points at
 * (i*h/k, j*h/k) for h = 1..k, each coordinate rounded the same way.  It is not
 * in the paper; it is the literal reading of the sum over harmonics h of the
 * point scaled by h/k, kept so that both readings can be checked.
 *
 * Every input element is converted to double exactly; every sum is formed in
 * double in ascending order of the stretch factor (or of h), which is the
 * order Eq. 2 adds the planes in.
 *
 * Parity pins (checked by the CPU test-suite, not by this file): HP_1 = FOP,
 * constant planes, linearity, gather/scatter adjointness, delta responses,
 * closed-form sums of injected harmonic signals, the touch counts of
 * Section IV-A and the loaded-points figures of Table II.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { HSO_F32 = 0, HSO_BF16 = 1, HSO_F16 = 2, HSO_F64 = 3 };
enum { HSO_STRETCH = 0, HSO_HFRAC = 1 };
enum { HSO_ZSYM = 0, HSO_ZFLOOR = 1 };

typedef struct {
    int64_t f;     /* bin j */
    int32_t z;     /* signed template index i */
    int32_t k;     /* harmonic level, 1-based */
    double power;  /* HP_k(i, j) */
} hso_cand;

/* ---- exact element conversion ------------------------------------------ */

static double half_bits_to_double(uint16_t h)
{
    /* IEEE 754 binary16: 1 sign, 5 exponent (bias 15), 10 fraction bits. */
    int sign = (h >> 15) & 1;
    int e = (h >> 10) & 0x1f;
    int frac = h & 0x3ff;
    double v;
    if (e == 0)
        v = ldexp((double)frac, -24);               /* subnormal or zero */
    else if (e == 31)
        v = frac ? NAN : INFINITY;
    else
        v = ldexp((double)(1024 + frac), e - 25);   /* (1 + f/1024) 2^(e-15) */
    return sign ? -v : v;
}

static double load_elem(const void *base, int dtype, size_t idx)
{
    switch (dtype) {
    case HSO_F32:
        return (double)((const float *)base)[idx];
    case HSO_F64:
        return ((const double *)base)[idx];
    case HSO_BF16: {
        /* bfloat16 is the top half of a binary32 */
        uint32_t bits = (uint32_t)((const uint16_t *)base)[idx] << 16;
        float f;
        memcpy(&f, &bits, sizeof f);
        return (double)f;
    }
    case HSO_F16:
        return half_bits_to_double(((const uint16_t *)base)[idx]);
    default:
        return NAN;
    }
}

/* ---- index maps ---------------------------------------------------------- */

/* floor(a / b) for b > 0 and any sign of a */
static int64_t floor_div(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0)
        q -= 1;
    return q;
}

/* Row of the input read for output row i when the plane is scaled by num/den
 * (Eq. 1 uses num = 1, den = k). */
static int64_t scale_row(int64_t i, int64_t num, int64_t den, int zround)
{
    if (zround == HSO_ZFLOOR)
        return floor_div(i * num, den);
    if (i >= 0)
        return (i * num) / den;
    return -((-i * num) / den);
}

/* Bin of the input read for output bin j (j >= 0). */
static int64_t scale_bin(int64_t j, int64_t num, int64_t den)
{
    return (j * num) / den;
}

static int check_shape(int nt, int64_t n)
{
    return (nt >= 1 && (nt % 2) == 1 && n >= 1) ? 0 : -1;
}

/* ---- Eq. 1: one stretch plane (gather form) ----------------------------- */

/* out[i+Z][j] = FOP(scale_row(i), scale_bin(j)) for every point of the plane,
 * scale = num/den with 1 <= num <= den.  Eq. 1 is num = 1, den = k. */
int hso_stretch(const void *fop, int dtype, int nt, int64_t n, int64_t num,
                int64_t den, int zround, double *out)
{
    if (check_shape(nt, n) || num < 1 || den < num)
        return -1;
    const int64_t Z = (nt - 1) / 2;
    for (int64_t i = -Z; i <= Z; ++i) {
        int64_t src_row = scale_row(i, num, den, zround) + Z;
        for (int64_t j = 0; j < n; ++j) {
            int64_t src_bin = scale_bin(j, num, den);
            out[(i + Z) * n + j] = load_elem(fop, dtype, (size_t)(src_row * n + src_bin));
        }
    }
    return 0;
}

/* ---- adjoint of Eq. 1 (scatter form, written from preimages) ------------ */

/* out[r+Z][b] = sum of w[i+Z][j] over every output point (i, j) whose Eq. 1
 * source is (r, b).  Written from the preimage of each source point rather
 * than from the forward map, so that gather/scatter adjointness checks one
 * against the other:
 *   bins: floor(j/k) = b  <=>  j in [k b, k b + k - 1];
 *   rows, floor rounding:     i in [k r, k r + k - 1];
 *   rows, symmetric rounding: r > 0: i in [k r, k r + k - 1];
 *                             r < 0: i in [k r - k + 1, k r];
 *                             r = 0: i in [-(k-1), k-1].                    */
int hso_stretch_adjoint(const double *w, int nt, int64_t n, int64_t k,
                        int zround, double *out)
{
    if (check_shape(nt, n) || k < 1)
        return -1;
    const int64_t Z = (nt - 1) / 2;
    for (int64_t r = -Z; r <= Z; ++r) {
        int64_t i_lo, i_hi;
        if (zround == HSO_ZFLOOR || r > 0) {
            i_lo = k * r;
            i_hi = k * r + k - 1;
        } else if (r < 0) {
            i_lo = k * r - k + 1;
            i_hi = k * r;
        } else {
            i_lo = -(k - 1);
            i_hi = k - 1;
        }
        if (i_lo < -Z) i_lo = -Z;
        if (i_hi > Z) i_hi = Z;
        for (int64_t b = 0; b < n; ++b) {
            int64_t j_lo = k * b, j_hi = k * b + k - 1;
            if (j_hi > n - 1) j_hi = n - 1;
            double acc = 0.0;
            for (int64_t i = i_lo; i <= i_hi; ++i)
                for (int64_t j = j_lo; j <= j_hi; ++j)
                    acc += w[(i + Z) * n + j];
            out[(r + Z) * n + b] = acc;
        }
    }
    return 0;
}

/* ---- Algorithm 1 order: materialised planes ------------------------------ */

/* hp[k-1][i+Z][j] for k = 1..H.
 * STRETCH: HP_1 = SP_1 = FOP; HP_k = HP_{k-1} + SP_k (Eq. 1 and Eq. 2), each
 *          stretch plane materialised first, as Algorithm 1 describes.
 * HFRAC:   S_k = sum over h = 1..k of the plane scaled by h/k, ascending h. */
int hso_planes(const void *fop, int dtype, int nt, int64_t n, int H,
               int index_mode, int zround, double *hp)
{
    if (check_shape(nt, n) || H < 1)
        return -1;
    const size_t plane = (size_t)nt * (size_t)n;
    double *sp = (double *)malloc(plane * sizeof(double));
    if (!sp)
        return -2;
    for (int k = 1; k <= H; ++k) {
        double *cur = hp + (size_t)(k - 1) * plane;
        if (index_mode == HSO_STRETCH) {
            hso_stretch(fop, dtype, nt, n, 1, k, zround, sp);
            for (size_t p = 0; p < plane; ++p)
                cur[p] = (k == 1) ? sp[p] : hp[(size_t)(k - 2) * plane + p] + sp[p];
        } else {
            for (size_t p = 0; p < plane; ++p)
                cur[p] = 0.0;
            for (int h = 1; h <= k; ++h) {
                hso_stretch(fop, dtype, nt, n, h, k, zround, sp);
                for (size_t p = 0; p < plane; ++p)
                    cur[p] += sp[p];
            }
        }
    }
    free(sp);
    return 0;
}

/* ---- per-point sums (the plain definition) ------------------------------- */

/* All H level values of output point (i, j), written to out[0..H-1]. */
static void point_levels(const void *fop, int dtype, int64_t Z, int64_t n, int H,
                         int index_mode, int zround, int64_t i, int64_t j,
                         double *out)
{
    if (index_mode == HSO_STRETCH) {
        double s = 0.0;
        for (int k = 1; k <= H; ++k) {
            int64_t r = scale_row(i, 1, k, zround) + Z;
            int64_t b = scale_bin(j, 1, k);
            s += load_elem(fop, dtype, (size_t)(r * n + b));
            out[k - 1] = s;
        }
    } else {
        for (int k = 1; k <= H; ++k) {
            double s = 0.0;
            for (int h = 1; h <= k; ++h) {
                int64_t r = scale_row(i, h, k, zround) + Z;
                int64_t b = scale_bin(j, h, k);
                s += load_elem(fop, dtype, (size_t)(r * n + b));
            }
            out[k - 1] = s;
        }
    }
}

/* Level values at a list of points: out[p*H + k-1]. */
int hso_sample(const void *fop, int dtype, int nt, int64_t n, int H,
               int index_mode, int zround, const int32_t *z, const int64_t *f,
               int64_t npts, double *out)
{
    if (check_shape(nt, n) || H < 1 || H > 64)
        return -1;
    const int64_t Z = (nt - 1) / 2;
    for (int64_t p = 0; p < npts; ++p) {
        if (z[p] < -Z || z[p] > Z || f[p] < 0 || f[p] >= n)
            return -1;
        point_levels(fop, dtype, Z, n, H, index_mode, zround, z[p], f[p], out + p * H);
    }
    return 0;
}

/* ---- Algorithm 2 order: detection ---------------------------------------- */

/* Loop order of Algorithm 2 (bins outer, templates, then levels), over the bin
 * range [f_lo, f_hi).  Every point whose level value exceeds TA(k, i)
 * (ta[(k-1)*nt + i+Z], binary32) is a candidate; up to cap of them are
 * written to cands.  Points within near_rel*|TA| of the threshold are also
 * listed in near (up to near_cap) so that callers comparing a lower-precision
 * result can exclude them.  Returns the true number of candidates, or -1 on
 * invalid arguments; *n_near receives the true number of near points. */
int64_t hso_detect(const void *fop, int dtype, int nt, int64_t n, int H,
                   int index_mode, int zround, const float *ta, double near_rel,
                   int64_t f_lo, int64_t f_hi, hso_cand *cands, int64_t cap,
                   hso_cand *near, int64_t near_cap, int64_t *n_near)
{
    if (check_shape(nt, n) || H < 1 || H > 64 || f_lo < 0 || f_hi > n || f_lo > f_hi)
        return -1;
    const int64_t Z = (nt - 1) / 2;
    double lv[64];
    int64_t nc = 0, nn = 0;
    for (int64_t j = f_lo; j < f_hi; ++j) {
        for (int64_t i = -Z; i <= Z; ++i) {
            point_levels(fop, dtype, Z, n, H, index_mode, zround, i, j, lv);
            for (int k = 1; k <= H; ++k) {
                double t = (double)ta[(size_t)(k - 1) * nt + (size_t)(i + Z)];
                double s = lv[k - 1];
                hso_cand c = { j, (int32_t)i, k, s };
                if (s > t) {
                    if (nc < cap)
                        cands[nc] = c;
                    ++nc;
                }
                if (fabs(s - t) <= near_rel * fabs(t)) {
                    if (nn < near_cap)
                        near[nn] = c;
                    ++nn;
                }
            }
        }
    }
    if (n_near)
        *n_near = nn;
    return nc;
}
