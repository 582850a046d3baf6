// Exact hypervolume of a point set (minimisation) with respect to a reference
// point: the measure of the union of the boxes [p, ref].  Used to score the
// approximation set (elitist archive) of the optimiser (Sec. 1 "approximation
// set", Sec. 2.4 archive of non-dominated solutions).
//
// Slicing on the last objective: HV_d(S) = sum over consecutive distinct
// values z_i of the last coordinate of (z_{i+1} - z_i) * HV_{d-1}({p in S:
// p_d <= z_i}), with z_{n+1} = ref_d; HV_2 by a sorted sweep; HV_1 = ref - min.
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/dmr.h"

namespace {

double hv2(std::vector<const double*>& pts, const double* ref) {
  std::sort(pts.begin(), pts.end(), [](const double* a, const double* b) {
    return a[0] < b[0] || (a[0] == b[0] && a[1] < b[1]);
  });
  double vol = 0.0, ybest = ref[1];
  for (size_t i = 0; i < pts.size(); ++i) {
    const double* p = pts[i];
    if (p[1] < ybest) {
      // horizontal strip [p.x, ref.x) x [p.y, ybest) joins the union
      vol += (ref[0] - p[0]) * (ybest - p[1]);
      ybest = p[1];
    }
  }
  return vol;
}

double hv_rec(std::vector<const double*> pts, const double* ref, int d) {
  if (pts.empty()) return 0.0;
  if (d == 1) {
    double m = ref[0];
    for (const double* p : pts) m = std::min(m, p[0]);
    return ref[0] - m;
  }
  if (d == 2) return hv2(pts, ref);
  std::sort(pts.begin(), pts.end(), [d](const double* a, const double* b) { return a[d - 1] < b[d - 1]; });
  double vol = 0.0;
  std::vector<const double*> active;
  for (size_t i = 0; i < pts.size(); ++i) {
    active.push_back(pts[i]);
    double z = pts[i][d - 1];
    double znext = (i + 1 < pts.size()) ? pts[i + 1][d - 1] : ref[d - 1];
    if (znext > z) vol += (znext - z) * hv_rec(active, ref, d - 1);
  }
  return vol;
}

}  // namespace

extern "C" int dmr_hypervolume(const double* pts, int n, int d, const double* ref, double* out) {
  if (!out || d < 1 || d > 6 || n < 0 || (n > 0 && !pts) || !ref) return DMR_EINVAL;
  std::vector<const double*> in;
  in.reserve(n);
  for (int i = 0; i < n; ++i) {
    const double* p = pts + (size_t)i * d;
    bool ok = true;
    for (int k = 0; k < d; ++k)
      if (!(p[k] < ref[k])) ok = false;  // outside the reference box (or NaN): no volume
    if (ok) in.push_back(p);
  }
  *out = hv_rec(in, ref, d);
  return DMR_OK;
}
