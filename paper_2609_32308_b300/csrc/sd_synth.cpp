// sd_synth.cpp -- seeded synthetic nearest-neighbour parameter sets.
//
// Input generation only: nothing here computes a loop energy or a design.
// The paper's Turner-2004 tables are not available, so callers without a
// parameter file get seeded synthetic integer tables (dcal/mol) with the
// shapes, signs, magnitudes and rotation symmetries of Turner-2004 dangle-0
// tables, written in the "SDENERGY 1" text format that sd_load_energy reads.
//
// Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast
// splittable pseudorandom number generators", OOPSLA 2014): a 64-bit counter
// advanced by 0x9E3779B97F4A7C15 and mixed by two xor-shift-multiply rounds.
// The test suite writes the same recipe in Python and checks that both give
// byte-identical files for the same seed.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

namespace {

struct SplitMix64 {
  uint64_t x;
  uint64_t next() {
    x += 0x9E3779B97F4A7C15ull;
    uint64_t z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  // integer in [lo, hi]
  int uniform(int lo, int hi) { return lo + (int)(next() % (uint64_t)(hi - lo + 1)); }
};

const char *kPairs[6] = {"AU", "CG", "GC", "UA", "GU", "UG"};
// helix strength of a pair type: GC/CG 3, AU/UA 2, GU/UG 1
int strength(int t) { return t == 1 || t == 2 ? 3 : t == 0 || t == 3 ? 2 : 1; }

void put_table(std::string &out, const char *name, const std::vector<int> &v) {
  out += name;
  out += " " + std::to_string(v.size()) + "\n";
  for (size_t k = 0; k < v.size(); k += 16) {
    for (size_t q = k; q < std::min(v.size(), k + 16); q++) {
      if (q > k) out += " ";
      out += std::to_string(v[q]);
    }
    out += "\n";
  }
}

// shortest decimal that reads back as the same double (Python's repr)
std::string shortest(double x) {
  char buf[64];
  for (int prec = 1; prec <= 17; prec++) {
    std::snprintf(buf, sizeof buf, "%.*g", prec, x);
    if (std::strtod(buf, nullptr) == x) break;
  }
  std::string s = buf;
  if (s.find_first_of(".e") == std::string::npos) s += ".0";
  return s;
}

}  // namespace

std::string sd_internal_synthetic_text(uint64_t seed) {
  SplitMix64 R{seed ^ 0x5D5D5D5D5D5D5D5Dull};
  std::string out = "SDENERGY 1\n";
  std::vector<int> stack(36);
  for (int t = 0; t < 6; t++)
    for (int s = t; s < 6; s++) {
      int v;
      if (strength(t) == 1 && strength(s) == 1) v = R.uniform(-150, 50);
      else v = -(50 * (strength(t) + strength(s)) - 50) - R.uniform(0, 100);
      stack[t * 6 + s] = stack[s * 6 + t] = v;
    }
  put_table(out, "stack", stack);
  for (const char *name : {"mismatch_hairpin", "mismatch_interior", "mismatch_interior_1n",
                           "mismatch_interior_23"}) {
    std::vector<int> m(96);
    for (int &x : m) x = R.uniform(-150, 0);
    put_table(out, name, m);
  }
  // int11[t][s][x][y] = int11[s][t][y][x]
  std::vector<int> i11(576);
  for (int t = 0; t < 6; t++)
    for (int s = 0; s < 6; s++)
      for (int x = 0; x < 4; x++)
        for (int y = 0; y < 4; y++) {
          const int here = ((t * 6 + s) * 4 + x) * 4 + y, mirror = ((s * 6 + t) * 4 + y) * 4 + x;
          i11[here] = mirror < here ? i11[mirror] : R.uniform(-100, 350);
        }
  put_table(out, "int11", i11);
  std::vector<int> i21(2304);
  for (int &x : i21) x = R.uniform(-100, 350);
  put_table(out, "int21", i21);
  // int22[t][s][a][b][c][d] = int22[s][t][c][d][a][b]
  std::vector<int> i22(9216);
  for (int t = 0; t < 6; t++)
    for (int s = 0; s < 6; s++)
      for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++)
          for (int c = 0; c < 4; c++)
            for (int d = 0; d < 4; d++) {
              const int here = ((((t * 6 + s) * 4 + a) * 4 + b) * 4 + c) * 4 + d;
              const int mirror = ((((s * 6 + t) * 4 + c) * 4 + d) * 4 + a) * 4 + b;
              i22[here] = mirror < here ? i22[mirror] : R.uniform(-100, 350);
            }
  put_table(out, "int22", i22);
  // loop-size tables: increasing from the first admissible size, 99999 below
  auto increasing = [&](const char *name, int lo, int hi, int first) {
    std::vector<int> v(31, 99999), xs;
    for (int k = first; k < 31; k++) xs.push_back(R.uniform(lo, hi));
    std::sort(xs.begin(), xs.end());
    std::copy(xs.begin(), xs.end(), v.begin() + first);
    put_table(out, name, v);
  };
  increasing("hairpin", 350, 650, 3);
  increasing("bulge", 280, 600, 1);
  increasing("interior", 100, 500, 2);
  std::vector<int> au(6);
  for (int t = 0; t < 6; t++) au[t] = strength(t) != 3 ? 50 : 0;
  put_table(out, "terminal_au", au);
  put_table(out, "ninio", {60});
  put_table(out, "max_ninio", {300});
  put_table(out, "ml_closing", {R.uniform(300, 400)});
  put_table(out, "ml_intern", {R.uniform(-100, 50)});
  put_table(out, "ml_base", {0});
  out += "lxc " + shortest(107.856) + "\n";
  const char *names[3] = {"triloop", "tetraloop", "hexaloop"};
  const int lens[3] = {5, 6, 8}, counts[3] = {20, 30, 4};
  for (int q = 0; q < 3; q++) {
    std::map<std::string, int> seen;  // ordered by sequence
    while ((int)seen.size() < counts[q]) {
      const int t = R.uniform(0, 5);
      std::string seq(1, kPairs[t][0]);
      for (int k = 0; k < lens[q] - 2; k++) seq += "ACGU"[R.uniform(0, 3)];
      seq += kPairs[t][1];
      if (!seen.count(seq)) seen[seq] = R.uniform(150, 500);
    }
    out += std::string(names[q]) + " " + std::to_string(seen.size()) + "\n";
    for (const auto &kv : seen) out += kv.first + " " + std::to_string(kv.second) + "\n";
  }
  return out;
}
