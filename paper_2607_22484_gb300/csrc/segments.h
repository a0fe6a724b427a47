// Splitting a solve's ordered product work into consecutive parts of about equal work:
// serving's large lane issues a fused solve as one launch per part. Pure host
// arithmetic, checked on the host by the tests.
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

namespace svt {

// Consecutive parts of `unit` (the work of each unit, in order) of about `target` work
// each, at most `max_parts`: the first unit of each part, then unit.size(). With
// parts = min(max_parts, max(1, ceil(total / target))) and per = total / parts, a part
// ends at the first unit where the running total reaches the next multiple of per, so
// every part holds at least one unit and at most per plus its last unit's work. An empty
// list gives {0, 0}.
inline std::vector<int> split_units(const std::vector<double> &unit, double target, int max_parts)
{
    const int nu = (int)unit.size();
    if (nu == 0)
        return {0, 0};
    double total = 0.0;
    for (double w : unit)
        total += w;
    const int want = (int)std::min<double>(std::max(1, max_parts),
                                           std::max(1.0, std::ceil(total / std::max(target, 1.0))));
    const double per = total / want;
    std::vector<int> bounds{0};
    double acc = 0.0;
    for (int i = 0; i < nu; ++i) {
        acc += unit[i];
        if (acc >= per * (double)bounds.size() && i + 1 < nu && (int)bounds.size() < want)
            bounds.push_back(i + 1);
    }
    bounds.push_back(nu);
    return bounds;
}

} // namespace svt
