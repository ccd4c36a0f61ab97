// Sweep levels of an unstructured mesh (host code only).
//
// The kinetic step's Gauss-Seidel sweep visits cells in a fixed order; on a
// structured grid the cells of one hyperplane i + j + k are independent and
// run in parallel.  On an unstructured mesh the equivalent schedule is a
// level per cell: in the order (key, index), each cell's level is one more
// than the highest level of its face neighbours that come before it (0 if
// none).  Face neighbours then never share a level, and every neighbour that
// precedes a cell in the sequential order lies on a lower level, so sweeping
// the levels in increasing order (cells of a level in any order, or at once)
// gives exactly the values of the sequential sweep; sweeping them in
// decreasing order gives those of the reverse sweep.  On a structured grid
// with key i + j + k the levels are the hyperplanes.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>
#include "../../include/gsis.h"

extern "C" gsis_status gsis_sweep_levels(int ncell, const int* offsets, const int* neighbours, const double* key,
                                         int* level, int* nlevels) {
    if (ncell < 0 || !nlevels || (ncell > 0 && (!offsets || !key || !level))) return GSIS_ERR_ARG;
    *nlevels = 0;
    if (ncell == 0) return GSIS_OK;
    if (offsets[0] != 0) return GSIS_ERR_ARG;
    for (int c = 0; c < ncell; ++c)
        if (offsets[c + 1] < offsets[c] || !std::isfinite(key[c])) return GSIS_ERR_ARG;
    if (offsets[ncell] > 0 && !neighbours) return GSIS_ERR_ARG;
    // neighbour lists: in range, no self-reference, symmetric
    std::vector<std::vector<int>> sorted(ncell);
    for (int c = 0; c < ncell; ++c) {
        for (int e = offsets[c]; e < offsets[c + 1]; ++e) {
            const int n = neighbours[e];
            if (n < 0 || n >= ncell || n == c) return GSIS_ERR_ARG;
            sorted[c].push_back(n);
        }
        std::sort(sorted[c].begin(), sorted[c].end());
    }
    for (int c = 0; c < ncell; ++c)
        for (int n : sorted[c])
            if (!std::binary_search(sorted[n].begin(), sorted[n].end(), c)) return GSIS_ERR_ARG;
    std::vector<int> order(ncell);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b] || (key[a] == key[b] && a < b); });
    std::vector<int> rank(ncell);
    for (int r = 0; r < ncell; ++r) rank[order[r]] = r;
    int top = 0;
    for (int r = 0; r < ncell; ++r) {
        const int c = order[r];
        int lv = 0;
        for (int n : sorted[c])
            if (rank[n] < r) lv = std::max(lv, level[n] + 1);
        level[c] = lv;
        top = std::max(top, lv);
    }
    *nlevels = top + 1;
    return GSIS_OK;
}
