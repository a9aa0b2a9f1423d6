// hs_post.cu -- the paper's candidate cap as a host post-step (Section IV-A):
// when a harmonic plane (level k) yields more than N_cand candidates, keep the
// first, the last or the largest N_cand of them.  "First" and "last" refer to
// the order in which Algorithm 2 visits the points: bins ascending, then
// templates z ascending (the level loop is innermost, so each level's
// candidates arrive in that (bin, z) order).  The kernels return every
// candidate in an unspecified order; this step makes the selection
// independent of how the GPU scheduled the work.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hs.h"

namespace {

thread_local std::string g_err;

struct Key {
    int k, z;
    uint32_t bin;
    float power;
    uint32_t idx;
};

Key key_of(const hs_cand &c, uint32_t i)
{
    Key k;
    k.k = (int)c.k;
    k.z = (int)c.z;
    k.bin = c.bin;
    k.power = c.power;
    k.idx = i;
    return k;
}

// Algorithm 2 visiting order within one level: bin, then z.
bool visit_before(const Key &a, const Key &b)
{
    return a.bin != b.bin ? a.bin < b.bin : a.z < b.z;
}

} // namespace

extern "C" {

const char *hs_postfilter_last_error(void) { return g_err.c_str(); }

hs_status hs_postfilter(const hs_cand *in, uint32_t n, int policy, uint32_t n_keep, hs_cand *out,
                        uint32_t *n_out)
{
    if ((!in && n > 0) || !n_out || (!out && n > 0)) {
        g_err = "null input, output or count";
        return HS_ERR_INVALID;
    }
    if (policy < HS_KEEP_FIRST || policy > HS_KEEP_LARGEST) {
        g_err = "unknown policy";
        return HS_ERR_INVALID;
    }
    if (out == in && n > 0) {
        g_err = "out must not alias in";
        return HS_ERR_INVALID;
    }
    std::vector<Key> keys(n);
    for (uint32_t i = 0; i < n; ++i)
        keys[i] = key_of(in[i], i);
    // group by level, each level in visiting order
    std::stable_sort(keys.begin(), keys.end(), [](const Key &a, const Key &b) {
        return a.k != b.k ? a.k < b.k : visit_before(a, b);
    });
    std::vector<Key> kept;
    kept.reserve(std::min<size_t>(n, (size_t)n_keep * 32));
    for (size_t lo = 0; lo < keys.size();) {
        size_t hi = lo;
        while (hi < keys.size() && keys[hi].k == keys[lo].k)
            ++hi;
        const size_t cnt = hi - lo, take = std::min<size_t>(cnt, n_keep);
        if (policy == HS_KEEP_FIRST) {
            kept.insert(kept.end(), keys.begin() + (long)lo, keys.begin() + (long)(lo + take));
        } else if (policy == HS_KEEP_LAST) {
            kept.insert(kept.end(), keys.begin() + (long)(hi - take), keys.begin() + (long)hi);
        } else { // largest power; equal powers: the later visited first
            std::vector<Key> g(keys.begin() + (long)lo, keys.begin() + (long)hi);
            std::partial_sort(g.begin(), g.begin() + (long)take, g.end(),
                              [](const Key &a, const Key &b) {
                                  if (a.power != b.power)
                                      return a.power > b.power;
                                  return visit_before(b, a);
                              });
            g.resize(take);
            std::sort(g.begin(), g.end(), visit_before);
            kept.insert(kept.end(), g.begin(), g.end());
        }
        lo = hi;
    }
    for (size_t i = 0; i < kept.size(); ++i)
        out[i] = in[kept[i].idx];
    *n_out = (uint32_t)kept.size();
    return HS_OK;
}

} // extern "C"
