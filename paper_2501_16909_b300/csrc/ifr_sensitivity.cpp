// Host reduction of colocation cells into slowdowns and a per-resource
// sensitivity vector.  The paper defines slowdown as colocated over isolated
// latency (Sec. 4.3, 4.4.1) and asks for constant interference during the
// victim's life (Sec. 4.1); the per-resource summary below is this library's
// reading (the paper gives no formula):
//   T = (last block exit - first block entry) / K per measurement
//   T0 = median of valid solo repeats; T[r][l] = median of valid repeats
//   slowdown = T / T0;  noise = (max - min) / median of solo repeats
//   S[r] = slowdown at the top level - 1;  AUC[r] = trapezoid of slowdown - 1
//   over the achieved intensity;  monotone[r]: no drop larger than 3 * noise.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/ifr.h"

namespace {

double median_of(std::vector<double> v) {
    if (v.empty()) return NAN;
    std::sort(v.begin(), v.end());
    const size_t n = v.size();
    return (n & 1) ? v[n / 2] : (v[n / 2 - 1] + v[n / 2]) / 2.0;
}

double per_launch_ns(const ifr_cell_result &c) {
    const int k = c.timing.repeats > 0 ? c.timing.repeats : 1;
    return ((double)c.timing.t_end_ns - (double)c.timing.t_start_ns) / (double)k;
}

}  // namespace

extern "C" int ifr_sensitivity(const ifr_cell_result *cells, size_t n, int victim, int n_stressors, int n_levels,
                               const double *intensity, ifr_sensitivity_out *out) {
    if (!out || (n > 0 && !cells) || n_stressors < 0 || n_stressors > IFR_MAX_STRESSORS || n_levels <= 0 ||
        n_levels > IFR_MAX_LEVELS)
        return IFR_ERR_ARG;
    memset(out, 0, sizeof *out);
    out->n_stressors = n_stressors;
    out->n_levels = n_levels;
    std::vector<double> solo;
    for (size_t i = 0; i < n; ++i) {
        const ifr_cell_result &c = cells[i];
        if (c.victim != victim || c.stressor >= 0) continue;
        if (c.valid) {
            solo.push_back(per_launch_ns(c));
            ++out->n_valid;
        } else {
            ++out->n_invalid;
        }
    }
    const double t0 = median_of(solo);
    out->t0_ns = t0;
    if (!solo.empty()) {
        const auto mm = std::minmax_element(solo.begin(), solo.end());
        out->noise = (*mm.second - *mm.first) / t0;
    } else {
        out->noise = NAN;
    }
    const int L = n_levels;
    for (int r = 0; r < n_stressors; ++r) {
        for (int l = 0; l <= L; ++l) {
            std::vector<double> ts;
            for (size_t i = 0; i < n; ++i) {
                const ifr_cell_result &c = cells[i];
                if (c.victim != victim || c.stressor != r || c.level != l) continue;
                if (c.valid) {
                    ts.push_back(per_launch_ns(c));
                    ++out->n_valid;
                } else {
                    ++out->n_invalid;
                }
            }
            out->slowdown[r][l] = ts.empty() ? NAN : median_of(ts) / t0;
        }
        for (int l = L + 1; l <= IFR_MAX_LEVELS; ++l) out->slowdown[r][l] = NAN;
        const double *row = out->slowdown[r];
        out->S[r] = row[L] - 1.0;
        bool any_nan = false;
        for (int l = 0; l <= L; ++l) any_nan |= std::isnan(row[l]);
        if (any_nan) {
            out->auc[r] = NAN;
            out->monotone[r] = 0;
            continue;
        }
        double a = 0.0;
        double x_prev = 0.0;
        int mono = 1;
        for (int l = 0; l < L; ++l) {
            const double x_next = intensity ? intensity[(size_t)r * L + l] : (double)(l + 1) / (double)L;
            a += (x_next - x_prev) * ((row[l] - 1.0) + (row[l + 1] - 1.0)) / 2.0;
            x_prev = x_next;
            if (!(row[l + 1] >= row[l] - 3.0 * out->noise)) mono = 0;
        }
        out->auc[r] = a;
        out->monotone[r] = mono;
    }
    for (int r = n_stressors; r < IFR_MAX_STRESSORS; ++r) {
        out->S[r] = NAN;
        out->auc[r] = NAN;
        for (int l = 0; l <= IFR_MAX_LEVELS; ++l) out->slowdown[r][l] = NAN;
    }
    return IFR_OK;
}
