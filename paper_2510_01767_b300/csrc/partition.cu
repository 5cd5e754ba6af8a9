// partition.cu -- load-balanced KD-tree partition with cutline refinement (Alg. 1, Sec. 3.1).
//
// Host code: the tree is grown best first on the workload L(B) = |C(B)| (the number of cameras
// assigned to a block), each node cut along the longer of the x / y extents of the coarse
// centres inside it, at a percentile q of those centres' coordinates that starts at the median
// and moves by bisection toward the lighter child for a few rounds. A box's cameras are those
// of its parent whose visibility ratio V (fast camera selection, Sec. 3.2) reaches tau; the
// ratios come from a caller-supplied function (on the GPU: lobe_fcs_coverage over the cameras'
// depth maps, one pass per tried cut).
//
// Readings (the paper leaves them open): boxes are half-open (lo <= p < hi); the percentile is
// the linear interpolation between the order statistics at (n - 1) q; after the bisection the
// children of the last evaluated cut are kept; among leaves of equal workload the earliest
// created is split first.
#include <algorithm>
#include <cmath>
#include <vector>

#include "lobe.h"

namespace {

struct Node {
    lobe_box_d box;
    std::vector<int32_t> cams;
    std::vector<int64_t> pts;  // indices of the centres inside the box
    long long serial;
};

// The q-quantile of sorted x by linear interpolation between the order statistics around
// (n - 1) q, the interpolation written from the end nearer t (so that t = 1 gives b exactly).
double quantile_linear(const std::vector<double> &x, double q)
{
    const size_t n = x.size();
    const double h = q * (double)(n - 1);
    double lo_f = std::floor(h);
    if (lo_f < 0) lo_f = 0;
    size_t i = (size_t)lo_f;
    if (i > n - 1) i = n - 1;
    const size_t j = i + 1 < n ? i + 1 : n - 1;
    const double t = h - lo_f;
    const double a = x[i], b = x[j], d = b - a;
    return t >= 0.5 ? b - d * (1.0 - t) : a + d * t;
}

bool inside(const double *p, const lobe_box_d &b)
{
    for (int k = 0; k < 3; ++k)
        if (!(p[k] >= b.lo[k] && p[k] < b.hi[k])) return false;
    return true;
}

}  // namespace

extern "C" lobe_status lobe_kd_partition(const double *centers, int64_t n, const lobe_box_d *root, int32_t n_cams,
                                         lobe_ratio_fn ratios, void *user, const lobe_kd_params *prm,
                                         lobe_box_d *leaves, uint8_t *leaf_cams)
{
    if (n < 0 || (n > 0 && !centers) || !root || n_cams < 0 || !ratios || !prm || !leaves ||
        (n_cams > 0 && !leaf_cams) || prm->n_blocks < 1 || prm->steps < 0)
        return LOBE_ERR_ARG;
    std::vector<double> V;

    // cameras of `parent` with V >= tau for each of the boxes
    auto cams_of = [&](const lobe_box_d *boxes, int nb, const std::vector<int32_t> &parent,
                       std::vector<int32_t> *out) -> bool {
        V.assign((size_t)n_cams * nb, 0.0);
        if (ratios(user, boxes, nb, V.data()) != 0) return false;
        for (int b = 0; b < nb; ++b) {
            out[b].clear();
            for (int32_t c : parent)
                if (V[(size_t)c * nb + b] >= prm->tau) out[b].push_back(c);
        }
        return true;
    };

    std::vector<Node> open;
    {
        Node r;
        r.box = *root;
        std::vector<int32_t> all(n_cams);
        for (int32_t c = 0; c < n_cams; ++c) all[c] = c;
        if (!cams_of(root, 1, all, &r.cams)) return LOBE_ERR_ARG;
        for (int64_t i = 0; i < n; ++i)
            if (inside(centers + 3 * i, r.box)) r.pts.push_back(i);
        r.serial = 0;
        open.push_back(std::move(r));
    }
    long long serial = 1;
    while ((int)open.size() < prm->n_blocks) {
        size_t best = 0;
        for (size_t i = 1; i < open.size(); ++i)
            if (open[i].cams.size() > open[best].cams.size() ||
                (open[i].cams.size() == open[best].cams.size() && open[i].serial < open[best].serial))
                best = i;
        Node node = std::move(open[best]);
        open.erase(open.begin() + (long)best);
        double ext[2] = {0.0, 0.0};
        if (!node.pts.empty())
            for (int d = 0; d < 2; ++d) {
                double mn = INFINITY, mx = -INFINITY;
                for (int64_t i : node.pts) {
                    mn = std::min(mn, centers[3 * i + d]);
                    mx = std::max(mx, centers[3 * i + d]);
                }
                ext[d] = mx - mn;
            }
        const int a = ext[0] >= ext[1] ? 0 : 1;
        std::vector<double> coords;
        coords.reserve(node.pts.size());
        for (int64_t i : node.pts) coords.push_back(centers[3 * i + a]);
        std::sort(coords.begin(), coords.end());
        double qlo = prm->q_lo, qhi = prm->q_hi, q = 0.5;
        lobe_box_d kids[2];
        std::vector<int32_t> kc[2];
        for (int s = 0; s < std::max(prm->steps, 1); ++s) {
            const double cut = coords.empty() ? 0.5 * (node.box.lo[a] + node.box.hi[a]) : quantile_linear(coords, q);
            kids[0] = node.box;
            kids[1] = node.box;
            kids[0].hi[a] = cut;
            kids[1].lo[a] = cut;
            if (!cams_of(kids, 2, node.cams, kc)) return LOBE_ERR_ARG;
            if (s + 1 >= prm->steps) break;
            if (kc[0].size() > kc[1].size()) {
                qhi = q;
                q = 0.5 * (qlo + q);
            } else if (kc[1].size() > kc[0].size()) {
                qlo = q;
                q = 0.5 * (qhi + q);
            } else {
                break;
            }
        }
        Node child[2];
        for (int k = 0; k < 2; ++k) {
            child[k].box = kids[k];
            child[k].cams = kc[k];
            child[k].serial = serial + k;
        }
        for (int64_t i : node.pts) child[inside(centers + 3 * i, kids[0]) ? 0 : 1].pts.push_back(i);
        open.push_back(std::move(child[0]));
        open.push_back(std::move(child[1]));
        serial += 2;
    }
    std::sort(open.begin(), open.end(), [](const Node &x, const Node &y) { return x.serial < y.serial; });
    for (size_t b = 0; b < open.size(); ++b) {
        leaves[b] = open[b].box;
        if (n_cams > 0) {
            std::fill(leaf_cams + b * n_cams, leaf_cams + (b + 1) * n_cams, (uint8_t)0);
            for (int32_t c : open[b].cams) leaf_cams[b * n_cams + c] = 1;
        }
    }
    return LOBE_OK;
}
