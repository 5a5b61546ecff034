// Trotter schedule: the op list of one second-order step.
//
// The paper integrates with a W^II evolution MPO (Sec. 2.5); with two-site
// gates the connectivity is handled the way Sec. 2.5 maps any graph onto the
// MPO path: bonds between path neighbours are applied directly, longer bonds
// after swap gates bring the two qubits next to each other.
//   forward half F = [even-position NN layer, odd-position NN layer,
//                     per long-range bond (i<j): swaps at j-1, j-2, ..., i+1,
//                     gate at (i, i+1), the swaps again in reverse order]
//   step = F(dt/2) then reversed(F)(dt/2); where the halves meet, mirrored
//   swaps cancel and the meeting gate layer runs once at dt.
// Every qubit's on-site Liouvillian is split over its bonds with weight 1/deg.
#include <algorithm>
#include <set>
#include <utility>

#include "internal.h"

namespace mpdo {

std::string build_schedule(int n, const std::vector<int>& bi, const std::vector<int>& bj,
                           std::vector<Layer>& layers, std::vector<double>& weights) {
    const int nb = (int)bi.size();
    if (nb < 1) return "need at least one bond";
    std::vector<int> deg(n, 0);
    std::set<std::pair<int, int>> seen;
    std::vector<std::pair<int, int>> bonds(nb);
    for (int k = 0; k < nb; ++k) {
        int i = bi[k], j = bj[k];
        if (i < 0 || j < 0 || i >= n || j >= n || i == j) return "bond " + std::to_string(k) + " is invalid";
        auto key = std::make_pair(std::min(i, j), std::max(i, j));
        if (!seen.insert(key).second) return "bond " + std::to_string(k) + " is a duplicate";
        bonds[k] = key;
        deg[i]++;
        deg[j]++;
    }
    for (int q = 0; q < n; ++q)
        if (deg[q] == 0) return "qubit " + std::to_string(q) + " is on no bond";
    weights.assign(n, 0.0);
    for (int q = 0; q < n; ++q) weights[q] = 1.0 / deg[q];

    // forward half
    std::vector<Layer> F;
    for (int parity = 0; parity < 2; ++parity) {
        Layer L;
        for (int k = 0; k < nb; ++k) {
            int i = bonds[k].first, j = bonds[k].second;
            if (j == i + 1 && (i % 2) == parity) L.push_back(Op{0, i, i, j, k, 0.5});
        }
        std::sort(L.begin(), L.end(), [](const Op& a, const Op& b) { return a.p < b.p; });
        if (!L.empty()) F.push_back(L);
    }
    for (int k = 0; k < nb; ++k) {
        int i = bonds[k].first, j = bonds[k].second;
        if (j == i + 1) continue;
        for (int p = j - 1; p >= i + 1; --p) F.push_back(Layer{Op{1, p, 0, 0, -1, 0.0}});
        F.push_back(Layer{Op{0, i, 0, 0, k, 0.5}});
        for (int p = i + 1; p <= j - 1; ++p) F.push_back(Layer{Op{1, p, 0, 0, -1, 0.0}});
    }
    // mirrored second half with junction cancellation / merge
    std::vector<Layer> R(F.rbegin(), F.rend());
    size_t fe = F.size(), rb = 0;
    auto same_positions = [](const Layer& a, const Layer& b) {
        if (a.size() != b.size()) return false;
        for (size_t t = 0; t < a.size(); ++t)
            if (a[t].p != b[t].p || a[t].kind != b[t].kind) return false;
        return true;
    };
    while (fe > 0 && rb < R.size() && F[fe - 1][0].kind == 1 && R[rb][0].kind == 1 &&
           same_positions(F[fe - 1], R[rb])) {
        --fe;
        ++rb;
    }
    if (fe == 0 || rb >= R.size() || F[fe - 1][0].kind != 0) return "internal: schedule junction";
    std::vector<Layer> seq(F.begin(), F.begin() + (fe - 1));
    Layer mid = F[fe - 1];
    for (auto& o : mid) o.frac = 1.0;
    seq.push_back(mid);
    for (size_t t = rb + 1; t < R.size(); ++t) seq.push_back(R[t]);

    // fill in which qubit sits where as the swaps move them
    std::vector<int> at(n);
    for (int q = 0; q < n; ++q) at[q] = q;
    for (auto& L : seq) {
        for (auto& o : L) {
            o.qa = at[o.p];
            o.qb = at[o.p + 1];
        }
        for (auto& o : L)
            if (o.kind == 1) std::swap(at[o.p], at[o.p + 1]);
    }
    for (int q = 0; q < n; ++q)
        if (at[q] != q) return "internal: schedule does not restore the path order";
    layers = seq;
    return "";
}

}  // namespace mpdo
