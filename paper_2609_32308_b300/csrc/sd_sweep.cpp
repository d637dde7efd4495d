// sd_sweep.cpp -- many values of lambda for one protein (Sec. 10 supported
// envelope and inverse-lambda tools).
//
// F*(p, lambda) = min_r E(r) + 100 lambda C(r) is the lower envelope of one
// line per synonymous design r, so it is concave and piecewise linear in
// lambda, and every linear piece is a design that is optimal for some lambda
// (a supported line).  The envelope is found by probing intersections: two
// adjacent supported lines meet at lambda* = (E2 - E1) / (100 (C1 - C2)); the
// exact design at lambda* either lies on both lines (lambda* is a
// breakpoint) or strictly below them (a new supported line between them).
// Every round probes all open intersections at once, as one batch of designs
// of the same protein (one lattice, one launch sequence), so the number of
// launch sequences grows with the depth of the search, not with the number
// of lines.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/sd.h"

namespace {

// the FP64 line of a design at lambda (kcal/mol), in dcal/mol
double line_at(const sd_result &r, double lam) { return (double)r.energy + 100.0 * lam * r.codon_cost; }

// Designs whose lines lie within the fixed-point rounding of the DP of each
// other (every codon cost is rounded to 2^-32 dcal/mol) are taken as equal.
double tie_tolerance(const sd_result &r) { return (r.n / 3 + 1) * std::ldexp(1.0, -31) + 1e-9; }

bool same_design(const sd_result &a, const sd_result &b) {
  return a.n == b.n && std::strcmp(a.mrna, b.mrna) == 0 && std::strcmp(a.structure, b.structure) == 0;
}

int run_batch(const sd_energy *E, const char *protein, const double *w,
              const std::vector<double> &lams, std::vector<sd_result> &out) {
  const int k = (int)lams.size();
  out.assign(k, sd_result{});
  std::vector<const char *> prots(k, protein);
  std::vector<int> st(k, SD_OK);
  int rc = sd_design_batch(E, k, prots.data(), w, 1, lams.data(), out.data(), st.data());
  if (rc != SD_OK) return rc;
  for (int q = 0; q < k; q++)
    if (st[q] != SD_OK) {
      for (auto &r : out) sd_result_free(&r);
      return st[q];
    }
  return SD_OK;
}

}  // namespace

extern "C" int sd_design_sweep(const sd_energy *energy, const char *protein,
                               const double *codon_weights, int k, const double *lambdas,
                               sd_result *outs, int *status) {
  if (!energy || !protein || !codon_weights || k < 0 || (k > 0 && (!lambdas || !outs || !status)))
    return SD_EINVAL;
  std::vector<const char *> prots(k, protein);
  return sd_design_batch(energy, k, prots.data(), codon_weights, 1, lambdas, outs, status);
}

extern "C" int sd_envelope(const sd_energy *energy, const char *protein,
                           const double *codon_weights, double lam_lo, double lam_hi,
                           int max_lines, sd_result *lines, double *breaks, int *count) {
  if (!energy || !protein || !codon_weights || !lines || !count || max_lines < 1 ||
      !(std::isfinite(lam_lo) && std::isfinite(lam_hi) && lam_lo >= 0.0 && lam_hi >= lam_lo))
    return SD_EINVAL;
  *count = 0;
  std::vector<sd_result> ends;
  std::vector<double> lams{lam_lo, lam_hi};
  int rc = run_batch(energy, protein, codon_weights, lams, ends);
  if (rc != SD_OK) return rc;
  // the envelope: lines in order of increasing lambda, closed[q] = the
  // intersection of lines q and q+1 is a known breakpoint
  std::vector<sd_result> L;
  std::vector<double> at;  // a lambda where each line is optimal
  std::vector<char> closed;
  std::vector<double> brk;
  L.push_back(ends[0]);
  at.push_back(lam_lo);
  if (same_design(ends[0], ends[1]) ||
      std::fabs(line_at(ends[0], lam_hi) - line_at(ends[1], lam_hi)) <= tie_tolerance(ends[0])) {
    sd_result_free(&ends[1]);
  } else {
    L.push_back(ends[1]);
    at.push_back(lam_hi);
  }
  closed.assign(L.size() > 1 ? L.size() - 1 : 0, 0);
  brk.assign(closed.size(), 0.0);
  bool capped = false;
  for (int round = 0; round < 64; round++) {
    std::vector<int> open;
    std::vector<double> probe;
    for (size_t q = 0; q + 1 < L.size(); q++) {
      if (closed[q]) continue;
      const double dc = L[q].codon_cost - L[q + 1].codon_cost;
      double x = dc > 0.0 ? (double)(L[q + 1].energy - L[q].energy) / (100.0 * dc) : at[q + 1];
      x = std::min(std::max(x, at[q]), at[q + 1]);
      open.push_back((int)q);
      probe.push_back(x);
    }
    if (open.empty()) break;
    if ((int)(L.size() + open.size()) > max_lines) {
      capped = true;
      break;
    }
    std::vector<sd_result> got;
    rc = run_batch(energy, protein, codon_weights, probe, got);
    if (rc != SD_OK) {
      for (auto &r : L) sd_result_free(&r);
      return rc;
    }
    // insert from the right so earlier indices stay valid
    for (int u = (int)open.size() - 1; u >= 0; u--) {
      const int q = open[u];
      const double x = probe[u];
      const double on_line = line_at(L[q], x);
      if (line_at(got[u], x) < on_line - tie_tolerance(got[u]) && !same_design(got[u], L[q]) &&
          !same_design(got[u], L[q + 1])) {
        L.insert(L.begin() + q + 1, got[u]);
        at.insert(at.begin() + q + 1, x);
        closed.insert(closed.begin() + q + 1, 0);
        brk.insert(brk.begin() + q + 1, 0.0);
      } else {
        sd_result_free(&got[u]);
        closed[q] = 1;
        brk[q] = x;
      }
    }
  }
  for (size_t q = 0; q < closed.size(); q++)
    if (!closed[q]) capped = true;
  // a line optimal at one lambda only (several designs tie at an end of the
  // range or at a breakpoint) supports no segment of the envelope: drop it
  if (!capped)
    for (size_t q = 0; q < L.size() && L.size() > 1;) {
      const double left = q == 0 ? lam_lo : brk[q - 1];
      const double right = q + 1 == L.size() ? lam_hi : brk[q];
      if (right > left) {
        q++;
        continue;
      }
      sd_result_free(&L[q]);
      L.erase(L.begin() + q);
      // the breakpoint to the right of the dropped line goes (the left one
      // stays and now joins its neighbours); the last line drops its left one
      if (q < brk.size()) brk.erase(brk.begin() + q);
      else if (!brk.empty()) brk.pop_back();
    }
  const int n = (int)L.size();
  for (int q = 0; q < n; q++) lines[q] = L[q];
  if (breaks)
    for (int q = 0; q + 1 < n; q++) breaks[q] = brk[q];
  *count = n;
  return capped ? SD_ESIZE : SD_OK;
}

extern "C" int sd_inverse_lambda(const sd_energy *energy, const char *protein,
                                 const double *codon_weights, double target_codon_cost,
                                 double lam_hi, double *lambda_out, sd_result *out) {
  if (!lambda_out || !out || !std::isfinite(target_codon_cost)) return SD_EINVAL;
  constexpr int kMax = 256;
  sd_result *lines = new (std::nothrow) sd_result[kMax];
  double *breaks = new (std::nothrow) double[kMax];
  if (!lines || !breaks) {
    delete[] lines;
    delete[] breaks;
    return SD_ENOMEM;
  }
  int count = 0;
  int rc = sd_envelope(energy, protein, codon_weights, 0.0, lam_hi, kMax, lines, breaks, &count);
  if (rc == SD_OK) {
    // lines come in increasing lambda, so with non-increasing codon cost:
    // the first line at or below the target starts the answer's interval
    int hit = -1;
    for (int q = 0; q < count && hit < 0; q++)
      if (lines[q].codon_cost <= target_codon_cost) hit = q;
    if (hit < 0) {
      rc = SD_EINFEASIBLE;
    } else {
      *lambda_out = hit == 0 ? 0.0 : breaks[hit - 1];
      *out = lines[hit];
      lines[hit].mrna = lines[hit].structure = nullptr;
    }
  }
  for (int q = 0; q < count; q++) sd_result_free(&lines[q]);
  delete[] lines;
  delete[] breaks;
  return rc;
}
