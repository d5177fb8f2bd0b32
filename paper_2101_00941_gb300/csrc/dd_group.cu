// Friends-of-friends grouping of single-pulse candidates (Sec. 2.2: the search reports one
// candidate per block and trial, so one pulse shows up at neighbouring DM trials, times and
// widths; grouping merges them). Host code: it runs on the few thousand candidates a chunk
// yields, after dd_candidates has sorted them.
//
//   DM of a candidate : dm_start + trial * dm_step of its range (FP64, one rounding per
//                       operation: the library's host code is built without FP contraction)
//   friends(a, b)     : |DM_a - DM_b| <= dm_link, and the boxcars [t, t + width) overlap or the
//                       later one starts at most t_link samples after the earlier one's last
//                       sample
//   groups            : connected components of the friendship graph
// Pairs are found by a sweep in order of t_start: a candidate's friends that start at or after
// it start no later than its last sample + t_link. Components are joined with a union-find, so
// the result does not depend on the order of the sweep.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "dd_internal.h"

namespace {

int64_t find_root(std::vector<int64_t>& parent, int64_t a) {
  while (parent[a] != a) {
    parent[a] = parent[parent[a]];
    a = parent[a];
  }
  return a;
}

}  // namespace

extern "C" {

int dd_group_candidates(const dd_cand_t* cands, int64_t n, const dd_range_t* ranges,
                        int32_t nranges, double dm_link, int64_t t_link, dd_group_t* out,
                        int64_t cap, int64_t* ngroups, int64_t* label) {
  if (!ngroups || n < 0 || cap < 0 || (n > 0 && (!cands || !ranges)) || (cap > 0 && !out) ||
      nranges < 1)
    return ddk::report_error(DD_ERR_ARG, "dd_group_candidates: bad argument");
  if (!(dm_link >= 0) || !std::isfinite(dm_link) || t_link < 0)
    return ddk::report_error(DD_ERR_ARG,
                             "dd_group_candidates: dm_link and t_link must be finite and >= 0");
  for (int64_t k = 0; k < n; ++k)
    if (cands[k].range < 0 || cands[k].range >= nranges || cands[k].width < 1)
      return ddk::report_error(DD_ERR_ARG,
                               "dd_group_candidates: a candidate's range or width is invalid");
  std::vector<double> dm(n);
  for (int64_t k = 0; k < n; ++k) {
    const dd_range_t& r = ranges[cands[k].range];
    const double step = (double)cands[k].trial * r.dm_step;
    dm[k] = r.dm_start + step;
  }
  std::vector<int64_t> order(n), parent(n);
  std::iota(order.begin(), order.end(), 0);
  std::iota(parent.begin(), parent.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    return cands[a].t_start < cands[b].t_start;
  });
  for (int64_t i = 0; i < n; ++i) {
    const int64_t a = order[i];
    const int64_t reach = cands[a].t_start + cands[a].width - 1 + t_link;
    for (int64_t j = i + 1; j < n && cands[order[j]].t_start <= reach; ++j) {
      const int64_t b = order[j];
      if (std::fabs(dm[a] - dm[b]) > dm_link) continue;
      const int64_t ra = find_root(parent, a), rb = find_root(parent, b);
      if (ra != rb) parent[std::max(ra, rb)] = std::min(ra, rb);
    }
  }
  // label = smallest index of the component (the root: unions always keep the smaller root)
  std::vector<int64_t> lab(n);
  for (int64_t k = 0; k < n; ++k) lab[k] = find_root(parent, k);
  int64_t g = 0;
  for (int64_t k = 0; k < n; ++k) {
    if (lab[k] != k) continue;
    if (g < cap) {
      dd_group_t& o = out[g];
      o.rep = k;
      o.members = 0;
      o.dm_lo = dm[k];
      o.dm_hi = dm[k];
      o.t_lo = cands[k].t_start;
      o.t_hi = cands[k].t_start + cands[k].width - 1;
    }
    ++g;
  }
  if (g <= cap) {
    // group records in order of their smallest index; index of each root's record
    std::vector<int64_t> slot(n, -1);
    int64_t s = 0;
    for (int64_t k = 0; k < n; ++k)
      if (lab[k] == k) slot[k] = s++;
    for (int64_t k = 0; k < n; ++k) {
      dd_group_t& o = out[slot[lab[k]]];
      o.members += 1;
      o.dm_lo = std::min(o.dm_lo, dm[k]);
      o.dm_hi = std::max(o.dm_hi, dm[k]);
      o.t_lo = std::min<int64_t>(o.t_lo, cands[k].t_start);
      o.t_hi = std::max<int64_t>(o.t_hi, cands[k].t_start + cands[k].width - 1);
      if (cands[k].snr > cands[o.rep].snr) o.rep = k;  // ties keep the smaller index
    }
  }
  if (label)
    for (int64_t k = 0; k < n; ++k) label[k] = lab[k];
  *ngroups = g;
  if (g > cap)
    return ddk::report_error(DD_ERR_CAP, "dd_group_candidates: more groups than the buffer");
  return DD_OK;
}

}  // extern "C"
