// Adaptive keyframe scheduler of CaRtGS (Sec. III-C.2, Eqs. 5-8), host side.
//
// Pool K of keyframes with remaining optimisation counts R and last losses L.
// add    : K, R, L grow by (v_{k+1}, r0, l) (Eqs. 5-7); l starts at +infinity.
// draw   : uniform choice among {i : r_i > 0} (the caller supplies the uniform
//          32-bit draw; the pick is draw mod count over the eligible keyframes in
//          pool order), then r_i -= 1.  When no keyframe is eligible the counts are
//          refilled first (Eq. 8): r_i = 2 for the d_k = max(1, floor(k / d))
//          largest losses (ties to the lower index), r_i = 1 otherwise.
// report : l_i <- the loss of the iteration that trained keyframe i.
#include <algorithm>
#include <limits>
#include <new>
#include <vector>

#include "cgs.h"

struct cgs_scheduler {
    int d;
    std::vector<int32_t> ids;
    std::vector<int32_t> r;
    std::vector<double> l;
};

namespace {

void refill(cgs_scheduler *s)
{
    const int k = (int)s->ids.size();
    const int dk = std::max(1, k / s->d);
    std::vector<int> order(k);
    for (int i = 0; i < k; i++) order[i] = i;
    // largest loss first; equal losses keep the lower index first
    std::stable_sort(order.begin(), order.end(), [s](int a, int b) { return s->l[a] > s->l[b]; });
    for (int i = 0; i < k; i++) s->r[i] = 1;
    for (int i = 0; i < dk && i < k; i++) s->r[order[i]] = 2;
}

}  // namespace

extern "C" {

cgs_scheduler *cgs_sched_create(int32_t d)
{
    if (d < 1) return nullptr;
    cgs_scheduler *s = new (std::nothrow) cgs_scheduler;
    if (s) s->d = d;
    return s;
}

void cgs_sched_destroy(cgs_scheduler *s) { delete s; }

int cgs_sched_add(cgs_scheduler *s, int32_t keyframe_id, int32_t r0)
{
    if (!s || r0 < 0) return CGS_ERR_ARG;
    s->ids.push_back(keyframe_id);
    s->r.push_back(r0);
    s->l.push_back(std::numeric_limits<double>::infinity());
    return (int)s->ids.size() - 1;
}

int cgs_sched_draw(cgs_scheduler *s, uint32_t rand_u32)
{
    if (!s || s->ids.empty()) return CGS_ERR_ARG;
    int count = 0;
    for (int32_t x : s->r) count += x > 0;
    if (count == 0) {
        refill(s);
        for (int32_t x : s->r) count += x > 0;
    }
    uint32_t pick = rand_u32 % (uint32_t)count;
    for (size_t i = 0; i < s->r.size(); i++) {
        if (s->r[i] > 0) {
            if (pick == 0) {
                s->r[i] -= 1;
                return (int)i;
            }
            pick--;
        }
    }
    return CGS_ERR_ARG;   // unreachable
}

int cgs_sched_report(cgs_scheduler *s, int32_t index, double loss)
{
    if (!s || index < 0 || index >= (int32_t)s->ids.size()) return CGS_ERR_ARG;
    s->l[index] = loss;
    return CGS_OK;
}

int cgs_sched_draw_n(cgs_scheduler *s, const uint32_t *rand_u32, int32_t n, int32_t *out)
{
    if (!s || n < 0 || (n > 0 && (!rand_u32 || !out))) return CGS_ERR_ARG;
    for (int32_t i = 0; i < n; i++) {
        const int rc = cgs_sched_draw(s, rand_u32[i]);
        if (rc < 0) return rc;
        out[i] = rc;
    }
    return CGS_OK;
}

int cgs_sched_report_n(cgs_scheduler *s, const int32_t *index, const double *loss, int32_t n)
{
    if (!s || n < 0 || (n > 0 && (!index || !loss))) return CGS_ERR_ARG;
    for (int32_t i = 0; i < n; i++) {
        const int rc = cgs_sched_report(s, index[i], loss[i]);
        if (rc != CGS_OK) return rc;
    }
    return CGS_OK;
}

int cgs_sched_state(const cgs_scheduler *s, int32_t *ids, int32_t *r, double *l, int32_t cap)
{
    if (!s) return CGS_ERR_ARG;
    const int k = (int)s->ids.size();
    for (int i = 0; i < k && i < cap; i++) {
        if (ids) ids[i] = s->ids[i];
        if (r) r[i] = s->r[i];
        if (l) l[i] = s->l[i];
    }
    return k;
}

}  // extern "C"
