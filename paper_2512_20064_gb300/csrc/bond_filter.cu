// Dynamic bond dimensions (Sec. 3.4.2) -- host code, no device work.
//
// The entanglement of an MPS grows from the edges to the centre, so a fixed
// bond dimension chi is redundant at the edges.  The filter keeps, at every
// bond, the least number of Schmidt coefficients whose discarded weight stays
// within the largest discarded weight that keeping chi coefficients incurs
// anywhere on the chain (or within a given budget): the maximum truncation
// error over the bonds is unchanged while the edge bonds shrink, and with them
// the per-site contraction cost 8 chi_l d chi_r.
//
// With align > 1 the kept counts are rounded up to a multiple of align (capped by chi and the
// spectrum length): more coefficients only lower the discarded weight, and bond dimensions that are
// multiples of the contraction tiles waste no tensor-core work on padding.
//
// Decisions are taken in FP64: T_c = sum_{j >= c} Lambda_j^2 is accumulated
// from the last coefficient towards c, and the discarded weight of keeping c
// of n coefficients is T_c / T_0.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/fastmps.h"

extern "C" int fastmps_bond_filter(int M, int d, const int *bond_in, const double *const *lambdas, int chi,
                                   double eps, int align, int *bond_out, double *discarded_out) {
    if (M < 1 || d < 2 || chi < 1 || align < 1 || !bond_in || !bond_out || (M > 1 && !lambdas))
        return FASTMPS_ERR_INVALID_ARG;
    if (bond_in[0] != 1 || bond_in[M] != 1) return FASTMPS_ERR_SHAPE;
    for (int k = 1; k < M; ++k)
        if (bond_in[k] < 1 || !lambdas[k - 1]) return FASTMPS_ERR_INVALID_ARG;
    // tail sums per bond: tails[k][c] = T_c of the coefficients right of site k (bond k+1)
    std::vector<std::vector<double>> tails(M > 1 ? M - 1 : 0);
    std::vector<int> cap(M > 1 ? M - 1 : 0);
    for (int k = 0; k + 1 < M; ++k) {
        const int n = bond_in[k + 1];
        std::vector<double> &T = tails[k];
        T.assign((size_t)n + 1, 0.0);
        double acc = 0.0;
        for (int j = n - 1; j >= 0; --j) {
            const double l = lambdas[k][j];
            acc += l * l;
            T[j] = acc;
        }
        if (!(T[0] > 0.0)) return FASTMPS_ERR_INVALID_ARG;
        cap[k] = std::min(chi, n);
    }
    double budget = eps;
    if (!(eps > 0.0)) {
        budget = 0.0;
        for (int k = 0; k + 1 < M; ++k) budget = std::max(budget, tails[k][cap[k]] / tails[k][0]);
    }
    bond_out[0] = 1;
    bond_out[M] = 1;
    for (int k = 0; k + 1 < M; ++k) {
        const std::vector<double> &T = tails[k];
        int keep = cap[k];
        for (int c = 1; c <= cap[k]; ++c)
            if (T[c] / T[0] <= budget) {
                keep = c;
                break;
            }
        if (align > 1) keep = std::min((keep + align - 1) / align * align, cap[k]);
        bond_out[k + 1] = keep;
    }
    // isometry shapes: d * chi_r >= chi_l at every site (left-to-right sweep)
    for (int k = 0; k + 1 < M; ++k) {
        const int need = (bond_out[k] + d - 1) / d;
        bond_out[k + 1] = std::min(std::max(bond_out[k + 1], need), cap[k]);
    }
    if (discarded_out) {
        discarded_out[0] = 0.0;
        discarded_out[M] = 0.0;
        for (int k = 0; k + 1 < M; ++k) discarded_out[k + 1] = tails[k][bond_out[k + 1]] / tails[k][0];
    }
    return FASTMPS_OK;
}
