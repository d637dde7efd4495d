// sd_host.cpp -- host side of libsd_b300: parameter loading, codon DFA
// construction, input validation, the exact-range check, device arenas for
// the packed tables, batch plans and the C ABI declared in include/sd.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <array>
#include <fstream>
#include <map>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/sd.h"
#include "sd_internal.h"

// ---------------------------------------------------------------------------
// energy parameters
// ---------------------------------------------------------------------------
std::string sd_internal_synthetic_text(uint64_t seed);  // sd_synth.cpp

struct sd_energy {
  std::string text;        // the parameter set in the "SDENERGY 1" text format
  SdParams h;              // host copy
  int32_t hairpin[31];     // raw hairpin length table (lengths 3..30)
  double lxc;              // long-hairpin extrapolation coefficient
  int32_t max_abs;         // largest |entry| over the entries the model reads
  SdParams *d = nullptr;   // device copy
  int device = 0;
};

namespace {

bool read_table(std::istream &in, const char *name, int32_t *dst, int count) {
  std::string word;
  int cnt = -1;
  if (!(in >> word >> cnt) || word != name || cnt != count) return false;
  for (int k = 0; k < count; k++)
    if (!(in >> dst[k])) return false;
  return true;
}

int nt_code(char c) {
  switch (c) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    case 'U': return 3;
    default: return -1;
  }
}

}  // namespace

extern "C" int sd_load_energy(const char *path_or_null, uint64_t synthetic_seed,
                              sd_energy **out) {
  if (!out) return SD_EINVAL;
  *out = nullptr;
  std::string text;
  if (path_or_null) {
    std::ifstream f(path_or_null);
    if (!f) return SD_EINVAL;
    std::ostringstream ss;
    ss << f.rdbuf();
    text = ss.str();
  } else {
    text = sd_internal_synthetic_text(synthetic_seed);
  }
  std::istringstream in(text);
  sd_energy *E = new (std::nothrow) sd_energy();
  if (!E) return SD_ENOMEM;
  E->text = text;
  SdParams &P = E->h;
  std::memset(&P, 0, sizeof(P));
  std::string word;
  int ver = 0;
  bool ok = (in >> word >> ver) && word == "SDENERGY" && ver == 1;
  int32_t mm[4][96];
  int32_t bulge[31], interior[31], one[5];
  ok = ok && read_table(in, "stack", &P.stack[0][0], 36);
  ok = ok && read_table(in, "mismatch_hairpin", mm[0], 96);
  ok = ok && read_table(in, "mismatch_interior", mm[1], 96);
  ok = ok && read_table(in, "mismatch_interior_1n", mm[2], 96);
  ok = ok && read_table(in, "mismatch_interior_23", mm[3], 96);
  ok = ok && read_table(in, "int11", &P.int11[0][0][0], 576);
  ok = ok && read_table(in, "int21", &P.int21[0][0][0], 2304);
  ok = ok && read_table(in, "int22", &P.int22[0][0][0], 9216);
  ok = ok && read_table(in, "hairpin", E->hairpin, 31);
  ok = ok && read_table(in, "bulge", bulge, 31);
  ok = ok && read_table(in, "interior", interior, 31);
  ok = ok && read_table(in, "terminal_au", P.au, 6);
  ok = ok && read_table(in, "ninio", &one[0], 1);
  ok = ok && read_table(in, "max_ninio", &one[1], 1);
  ok = ok && read_table(in, "ml_closing", &one[2], 1);
  ok = ok && read_table(in, "ml_intern", &one[3], 1);
  ok = ok && read_table(in, "ml_base", &one[4], 1);
  ok = ok && (in >> word >> E->lxc) && word == "lxc" && std::isfinite(E->lxc);
  const char *names[3] = {"triloop", "tetraloop", "hexaloop"};
  const int lens[3] = {5, 6, 8};
  for (int s = 0; s < 3 && ok; s++) {
    int cnt = -1;
    ok = (in >> word >> cnt) && word == names[s] && cnt >= 0 && cnt <= 64;
    P.nspecial[s] = ok ? cnt : 0;
    for (int k = 0; k < P.nspecial[s] && ok; k++) {
      std::string seq;
      int e = 0;
      ok = (in >> seq >> e) && (int)seq.size() == lens[s];
      int code = 0;
      for (int q = 0; q < lens[s] && ok; q++) {
        int c = nt_code(seq[q]);
        ok = c >= 0;
        code |= (c < 0 ? 0 : c) << (2 * q);
      }
      P.special_code[s][k] = code;
      P.special_e[s][k] = e;
    }
  }
  if (!ok) {
    delete E;
    return SD_EINVAL;
  }
  std::memcpy(P.mmH, mm[0], sizeof(mm[0]));
  std::memcpy(P.mmI, mm[1], sizeof(mm[1]));
  std::memcpy(P.mm1n, mm[2], sizeof(mm[2]));
  std::memcpy(P.mm23, mm[3], sizeof(mm[3]));
  for (int k = 0; k < 31; k++) {
    P.bulge[k] = bulge[k];
    P.interior[k] = interior[k];
  }
  P.ninio = one[0];
  P.maxninio = one[1];
  P.mlclosing = one[2];
  P.mlintern = one[3];
  P.mlbase = one[4];
  // magnitude of every entry the model can read (loop-size tables from
  // their smallest admissible size), for the exact-range check
  int32_t mx = 0;
  auto acc = [&](const int32_t *p, int cnt) {
    for (int k = 0; k < cnt; k++) mx = std::max(mx, std::abs(p[k]));
  };
  acc(&P.stack[0][0], 36);
  acc(&P.mmH[0][0], 4 * 96);
  acc(&P.int11[0][0][0], 576 + 2304 + 9216);
  acc(E->hairpin + 3, 28);
  acc(P.bulge + 1, 30);
  acc(P.interior + 2, 29);
  acc(P.au, 6);
  acc(one, 5);
  for (int s = 0; s < 3; s++) acc(P.special_e[s], P.nspecial[s]);
  E->max_abs = mx;
  if (mx > 100000) {
    delete E;
    return SD_EINVAL;
  }
  // lower bound of every two-loop energy of size (l1, l2)
  for (int l1 = 0; l1 <= SD_MAXTWO; l1++)
    for (int l2 = 0; l2 <= SD_MAXTWO; l2++) {
      int lb = 0;
      if (l1 + l2 <= SD_MAXTWO) {
        lb = 1 << 30;
        for (int t = 0; t < 6; t++)
          for (int ti = 0; ti < 6; ti++)
            for (int x = 0; x < 256; x++)
              lb = std::min(lb, sd_twoloop_energy(P, t, ti, l1, l2, x >> 6, (x >> 4) & 3,
                                                  (x >> 2) & 3, x & 3));
      }
      P.lb2[l1][l2] = lb;
    }
  if (cudaGetDevice(&E->device) != cudaSuccess) {
    delete E;
    return SD_ECUDA;
  }
  if (cudaMalloc(&E->d, sizeof(SdParams)) != cudaSuccess) {
    delete E;
    return SD_ECUDA;
  }
  if (cudaMemcpy(E->d, &P, sizeof(SdParams), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(E->d);
    delete E;
    return SD_ECUDA;
  }
  *out = E;
  return SD_OK;
}

extern "C" int sd_energy_save(const sd_energy *e, const char *path) {
  if (!e || !path) return SD_EINVAL;
  std::ofstream f(path, std::ios::binary);
  if (!f) return SD_EINVAL;
  f << e->text;
  return f.good() ? SD_OK : SD_EINVAL;
}

extern "C" void sd_energy_free(sd_energy *e) {
  if (!e) return;
  if (e->d) cudaFree(e->d);
  delete e;
}

// ---------------------------------------------------------------------------
// codon DFA (Sec. 3): a trie per amino acid between single codon-boundary
// states, the whole -ln w on the third edge
// ---------------------------------------------------------------------------
namespace {

// standard genetic code in the textbook U C A G layout
char translate(int x, int y, int z) {
  static const char tbl[] =
      "FFLLSSSSYY**CC*W"
      "LLLLPPPPHHQQRRRR"
      "IIIMTTTTNNKKSSRR"
      "VVVVAAAADDEEGGGG";
  static const int ucag[4] = {2, 1, 3, 0};  // A C G U -> position in U C A G
  return tbl[16 * ucag[x] + 4 * ucag[y] + ucag[z]];
}

struct HostLattice {
  int n = 0, N = 0, E = 0;
  int width = 0;                // most states on one layer
  int maxin = SD_MAXIN;         // stride of the in-edge lists
  std::vector<int32_t> lstart, layer;
  std::vector<SdEdge> out, in;  // N*SD_MAXOUT, N*maxin
  std::vector<uint8_t> out_cnt, in_cnt, in_mask, out_mask;
  std::vector<int32_t> e_from, e_to, e_label;  // (from, label) order
  std::vector<int64_t> e_cost;
  double qmax_sum = 0.0;  // sum over codon positions of the largest codon cost (FP64)
  std::vector<int32_t> caps;  // room of each candidate list (empty: worst case)
  int layout = SD_LAYOUT_SPAN;  // layout of the full tables
};

// Entries of each full table in a layout (see SdDesign::layout); wclass is
// the layer width of the kernel instance the plan runs (slots per cell).
int64_t table_cells(const HostLattice &L, int wclass) {
  const int64_t n = L.n, N = L.N;
  if (L.layout == SD_LAYOUT_SQUARE) return N * N;
  if (L.layout == SD_LAYOUT_PACKED) {
    int64_t c = 0;
    for (int v = 0; v < N; v++) c += N - L.lstart[L.layer[v] + 1];
    return c;
  }
  return n * (n + 1) / 2 * wclass * wclass;
}

// Row offsets of the forward-packed layout.
std::vector<int64_t> packed_offsets(const HostLattice &L) {
  std::vector<int64_t> off(L.N);
  int64_t c = 0;
  for (int v = 0; v < L.N; v++) {
    off[v] = c;
    c += L.N - L.lstart[L.layer[v] + 1];
  }
  return off;
}

// worst-case room of C_b: every state at least five layers before b
int32_t worst_room(const HostLattice &L, int v) { return L.lstart[std::max(0, L.layer[v] - 4)]; }
int32_t room(const HostLattice &L, int v) {
  return L.caps.empty() ? worst_room(L, v) : std::min(L.caps[v], worst_room(L, v));
}

int64_t codon_fx(double lambda, double w) {
  const double lam100 = 100.0 * lambda;
  const double q = -std::log(w);
  const double x = lam100 * q;
  return (int64_t)std::llrint(std::ldexp(x, 32));
}

struct E3 {
  int from, to, label;
  int64_t cost;
};

// Forbidden-motif automaton (Sec. 3: the Aho-Corasick automaton of the motif
// set, complete over A C G U): its states are the distinct prefixes of the
// motifs, numbered by (length, sequence); go[m][c] is the longest suffix of
// prefix(m) + c that is again a prefix; bad[m] marks the states whose prefix
// ends with a motif (a transition into one of them completes a motif).
struct MotifAutomaton {
  std::vector<std::string> pre;
  std::vector<std::array<int, 4>> go;
  std::vector<char> bad;
  int build(const std::vector<std::string> &motifs) {
    std::vector<std::string> all{""};
    for (const auto &m : motifs)
      for (size_t l = 1; l <= m.size(); l++) all.push_back(m.substr(0, l));
    std::sort(all.begin(), all.end(), [](const std::string &a, const std::string &b) {
      return a.size() != b.size() ? a.size() < b.size() : a < b;
    });
    all.erase(std::unique(all.begin(), all.end()), all.end());
    pre = all;
    std::map<std::string, int> id;
    for (size_t k = 0; k < pre.size(); k++) id[pre[k]] = (int)k;
    go.assign(pre.size(), {0, 0, 0, 0});
    bad.assign(pre.size(), 0);
    for (size_t k = 0; k < pre.size(); k++) {
      for (const auto &m : motifs)
        if (pre[k].size() >= m.size() && pre[k].compare(pre[k].size() - m.size(), m.size(), m) == 0)
          bad[k] = 1;
      for (int c = 0; c < 4; c++) {
        std::string t = pre[k] + "ACGU"[c];
        while (!id.count(t)) t.erase(0, 1);
        go[k][c] = id[t];
      }
    }
    return (int)pre.size();
  }
};

// The product of a layered DFA (states by layer, edges) with the motif
// automaton: states (q, m) reachable from (source, root) without entering a
// bad m, the last layer's states merged into one sink, trimmed to the states
// that reach the sink, numbered layer by layer and by (q, m) inside a layer.
// Returns SD_OK or SD_EINFEASIBLE (no motif-free design).
int motif_product(int n, const std::vector<int32_t> &layer_of, const std::vector<E3> &edges,
                  const MotifAutomaton &M, std::vector<int32_t> &nlayer, std::vector<E3> &nedges) {
  const int N0 = (int)layer_of.size();
  std::vector<std::vector<int>> outs(N0);
  for (size_t e = 0; e < edges.size(); e++) outs[edges[e].from].push_back((int)e);
  // forward: product states per layer, keyed by (q, m)
  std::vector<std::map<std::pair<int, int>, int>> at(n + 1);
  std::vector<std::pair<int, int>> st;  // product state -> (q, m)
  std::vector<int> st_layer;
  struct PE {
    int from, to, label;
    int64_t cost;
  };
  std::vector<PE> pe;
  auto state = [&](int l, int q, int m) {
    auto it = at[l].find({q, m});
    if (it != at[l].end()) return it->second;
    const int id = (int)st.size();
    at[l][{q, m}] = id;
    st.push_back({q, m});
    st_layer.push_back(l);
    return id;
  };
  state(0, 0, 0);
  for (int l = 0; l < n; l++) {
    std::vector<std::pair<std::pair<int, int>, int>> cur(at[l].begin(), at[l].end());
    for (const auto &kv : cur) {
      const int q = kv.first.first, m = kv.first.second;
      for (int e : outs[q]) {
        const int m2 = M.go[m][edges[e].label];
        if (M.bad[m2]) continue;
        const int t = state(l + 1, edges[e].to, l + 1 == n ? 0 : m2);
        pe.push_back({kv.second, t, edges[e].label, edges[e].cost});
      }
    }
  }
  if (at[n].empty()) return SD_EINFEASIBLE;
  // backward: keep states that reach the sink
  const int P = (int)st.size();
  std::vector<char> live(P, 0);
  live[at[n].begin()->second] = 1;
  std::vector<std::vector<int>> pin(P);
  for (size_t e = 0; e < pe.size(); e++) pin[pe[e].to].push_back((int)e);
  for (int l = n; l >= 1; l--)
    for (const auto &kv : at[l])
      if (live[kv.second])
        for (int e : pin[kv.second]) live[pe[e].from] = 1;
  if (!live[0]) return SD_EINFEASIBLE;
  // numbering: layer by layer, (q, m) order inside a layer (map order)
  std::vector<int> nid(P, -1);
  nlayer.clear();
  for (int l = 0; l <= n; l++)
    for (const auto &kv : at[l])
      if (live[kv.second]) {
        nid[kv.second] = (int)nlayer.size();
        nlayer.push_back(l);
      }
  nedges.clear();
  for (const auto &e : pe)
    if (live[e.from] && live[e.to]) nedges.push_back({nid[e.from], nid[e.to], e.label, e.cost});
  return SD_OK;
}

int build_lattice(const char *protein, const double *w, double lambda, HostLattice &L,
                  const MotifAutomaton *motifs = nullptr) {
  const int A = (int)std::strlen(protein);
  for (int k = 0; k < A; k++)
    if (protein[k] == '*' && k != A - 1) return SD_EINVAL;
  L.n = 3 * A;
  L.lstart.assign(L.n + 2, 0);
  L.layer.clear();
  std::vector<E3> edges;
  L.layer.push_back(0);
  int boundary = 0;
  L.qmax_sum = 0.0;
  for (int k = 0; k < A; k++) {
    const char aa = protein[k];
    bool used[4][4][4] = {};
    int cnt = 0;
    double wmax = 0.0, qmax = 0.0;
    for (int x = 0; x < 4; x++)
      for (int y = 0; y < 4; y++)
        for (int z = 0; z < 4; z++) {
          if (translate(x, y, z) != aa) continue;
          const double ww = w[16 * x + 4 * y + z];
          if (!(ww > 0.0 && ww <= 1.0)) return SD_EINVAL;
          used[x][y][z] = true;
          cnt++;
          wmax = std::max(wmax, ww);
          qmax = std::max(qmax, (100.0 * lambda) * -std::log(ww));
        }
    if (cnt == 0 || wmax != 1.0) return SD_EINVAL;
    L.qmax_sum += qmax;
    int first[4], pre[4][4];
    L.lstart[3 * k + 1] = (int)L.layer.size();
    for (int x = 0; x < 4; x++) {
      first[x] = -1;
      bool any = false;
      for (int y = 0; y < 4; y++)
        for (int z = 0; z < 4; z++) any |= used[x][y][z];
      if (any) {
        first[x] = (int)L.layer.size();
        L.layer.push_back(3 * k + 1);
      }
    }
    L.lstart[3 * k + 2] = (int)L.layer.size();
    for (int x = 0; x < 4; x++)
      for (int y = 0; y < 4; y++) {
        pre[x][y] = -1;
        bool any = false;
        for (int z = 0; z < 4; z++) any |= used[x][y][z];
        if (any) {
          pre[x][y] = (int)L.layer.size();
          L.layer.push_back(3 * k + 2);
        }
      }
    L.lstart[3 * k + 3] = (int)L.layer.size();
    const int next = (int)L.layer.size();
    L.layer.push_back(3 * k + 3);
    for (int x = 0; x < 4; x++)
      if (first[x] >= 0) edges.push_back({boundary, first[x], x, 0});
    for (int x = 0; x < 4; x++)
      for (int y = 0; y < 4; y++)
        if (pre[x][y] >= 0) edges.push_back({first[x], pre[x][y], y, 0});
    for (int x = 0; x < 4; x++)
      for (int y = 0; y < 4; y++)
        for (int z = 0; z < 4; z++)
          if (used[x][y][z])
            edges.push_back({pre[x][y], next, z, codon_fx(lambda, w[16 * x + 4 * y + z])});
    boundary = next;
  }
  if (motifs) {
    std::vector<int32_t> nlayer;
    std::vector<E3> nedges;
    const int rc = motif_product(L.n, L.layer, edges, *motifs, nlayer, nedges);
    if (rc != SD_OK) return rc;
    L.layer = nlayer;
    edges = nedges;
    for (int l = 0, v = 0; l <= L.n + 1; l++) {
      while (v < (int)L.layer.size() && L.layer[v] < l) v++;
      L.lstart[l] = v;
    }
  }
  L.N = (int)L.layer.size();
  L.lstart[L.n + 1] = L.N;
  L.E = (int)edges.size();
  L.width = 0;
  for (int l = 0; l <= L.n; l++) L.width = std::max(L.width, L.lstart[l + 1] - L.lstart[l]);
  if (L.width > SD_W_WIDE) return SD_ESIZE;
  std::vector<int> indeg(L.N, 0);
  int maxdeg = 0;
  for (const auto &e : edges) maxdeg = std::max(maxdeg, ++indeg[e.to]);
  if (maxdeg > SD_MAXIN_WIDE) return SD_ESIZE;
  L.maxin = L.width <= SD_W && maxdeg <= SD_MAXIN ? SD_MAXIN : SD_MAXIN_WIDE;
  L.out.assign((size_t)L.N * SD_MAXOUT, SdEdge{-1, -1, 0});
  L.in.assign((size_t)L.N * L.maxin, SdEdge{-1, -1, 0});
  L.out_cnt.assign(L.N, 0);
  L.in_cnt.assign(L.N, 0);
  L.in_mask.assign(L.N, 0);
  L.out_mask.assign(L.N, 0);
  std::vector<int> ord(edges.size());
  for (size_t e = 0; e < edges.size(); e++) ord[e] = (int)e;
  std::sort(ord.begin(), ord.end(), [&](int p, int q) {
    if (edges[p].from != edges[q].from) return edges[p].from < edges[q].from;
    return edges[p].label < edges[q].label;
  });
  for (int e : ord) {
    const E3 &x = edges[e];
    if (L.out_cnt[x.from] >= SD_MAXOUT) return SD_EINVAL;
    L.out[(size_t)x.from * SD_MAXOUT + L.out_cnt[x.from]++] = SdEdge{x.to, x.label, x.cost};
    L.out_mask[x.from] |= 1 << x.label;
    L.e_from.push_back(x.from);
    L.e_to.push_back(x.to);
    L.e_label.push_back(x.label);
    L.e_cost.push_back(x.cost);
  }
  std::sort(ord.begin(), ord.end(), [&](int p, int q) {
    if (edges[p].to != edges[q].to) return edges[p].to < edges[q].to;
    if (edges[p].label != edges[q].label) return edges[p].label < edges[q].label;
    return edges[p].from < edges[q].from;
  });
  for (int e : ord) {
    const E3 &x = edges[e];
    if (L.in_cnt[x.to] >= L.maxin) return SD_EINVAL;
    L.in[(size_t)x.to * L.maxin + L.in_cnt[x.to]++] = SdEdge{x.from, x.label, x.cost};
    L.in_mask[x.to] |= 1 << x.label;
  }
  return SD_OK;
}

// Exact-range check: every partial-structure value must stay below 2^57 in
// magnitude.  A structure on n nucleotides has at most n/2 + 1 loops, each of
// at most 5 table entries plus the long-hairpin extrapolation.
int range_check(const sd_energy *E, const HostLattice &L) {
  const double n = L.n;
  double lx = n > 30 ? std::fabs(E->lxc * std::log(n / 30.0)) : 0.0;
  double ebound = (n / 2.0 + 1.0) * (5.0 * E->max_abs + lx + 1.0);
  double total = std::ldexp(ebound, 32) + std::ldexp(L.qmax_sum, 32) + std::ldexp(n, 32);
  return total < std::ldexp(1.0, 57) ? SD_OK : SD_ERANGE;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// ---------------------------------------------------------------------------
// plans
// ---------------------------------------------------------------------------
struct PlanItem {
  std::string protein;
  double lambda = 0.0;
  double w[64];
  HostLattice L;
  int status = SD_OK;
  int dev_index = -1;  // position in the device design array
  SdDesign d{};        // device pointers (host copy of the struct)
  int regrows = 0;     // runs repeated because a presized candidate list overflowed
  int32_t *own_cand = nullptr;  // worst-case candidate room allocated by a regrow
  double pred_visits = -1.0;    // predicted candidate visits of the S2 scans (< 0: none)
};

// Designs of a plan that run on one stream of a multi-stream schedule.
struct PlanBin {
  std::vector<int> dev;           // device indices of the plan, non-increasing n
  std::vector<int> ns;
  std::vector<int32_t> cpre;
  SdDesign *d_designs = nullptr;  // copies of the plan's records, in bin order
  int32_t *d_cpre = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
};

struct sd_plan {
  const sd_energy *energy = nullptr;
  std::vector<PlanItem> items;
  std::vector<SdDesign> hdesigns;
  SdDesign *d_designs = nullptr;
  char *arena = nullptr;
  size_t arena_bytes = 0;
  int max_n = 0;
  int64_t launches = 0;
  cudaStream_t last_stream = nullptr;
  int group = 32;  // threads per layer pair in the fill
  std::vector<int> ns;            // lengths in device order (non-increasing)
  std::vector<int32_t> cpre_host; // prefix sums of ns + 1
  int32_t *d_cpre = nullptr;
  // CUDA graph of one whole run (captured on first use when enabled)
  bool use_graph = false;
  bool graph_timed = false;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int64_t graph_launches = 0;
  bool timing = false;
  bool timed_run = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // multi-stream schedule (sd_plan_set_streams): bins run concurrently
  std::vector<PlanBin> bins;
  cudaEvent_t fork = nullptr;
  int wclass = SD_W;  // layer width of the kernel instance (SD_W or SD_W_WIDE)
};

// the kernel instance of a plan's layer width
static int k_run(const sd_plan *p, const SdDesign *d, int count, const int *ns, const int32_t *cpre,
                 cudaStream_t st, int64_t *launches, void *const *events) {
  return p->wclass == SD_W
             ? sd_k_run(d, count, ns, cpre, p->energy->d, st, launches, events, p->group)
             : sd_k_run_wide(d, count, ns, cpre, p->energy->d, st, launches, events, 32);
}

namespace {

struct Carver {
  char *base;
  size_t off = 0;
  template <class T>
  T *take(size_t count) {
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off = align_up(off + count * sizeof(T));
    return p;
  }
};

// lay out one design's buffers (base == nullptr: only measure) for the
// kernel instance of layer width wclass
size_t carve(char *base, const HostLattice &L, SdDesign &d, int wclass) {
  Carver c{base};
  const int64_t n = L.n, N = L.N;
  const int64_t ncell = n * (n + 1) / 2;
  int64_t cap = 0;
  for (int v = 0; v < N; v++) cap += room(L, v);
  d.n = (int)n;
  d.N = (int)N;
  d.ncell = ncell;
  d.layout = L.layout;
  d.table_cells = table_cells(L, wclass);
  d.maxin = L.maxin;
  d.lstart = c.take<int32_t>(n + 2);
  d.layer = c.take<int32_t>(N);
  d.pos = c.take<int32_t>(N);
  d.out = c.take<SdEdge>(N * SD_MAXOUT);
  d.out_cnt = c.take<uint8_t>(N);
  d.in = c.take<SdEdge>(N * L.maxin);
  d.in_cnt = c.take<uint8_t>(N);
  d.in_mask = c.take<uint8_t>(N);
  d.out_mask = c.take<uint8_t>(N);
  d.hp_len = c.take<int32_t>(n + 1);
  d.fo = c.take<SdFlatEdge>(std::max(L.E, 1));
  d.fo_off = c.take<int32_t>(N + 1);
  d.fi = c.take<SdFlatEdge>(std::max(L.E, 1));
  d.fi_off = c.take<int32_t>(N + 1);
  const size_t ring = (size_t)SD_RING * (n + 1) * wclass * wclass;
  const int64_t tc = std::max<int64_t>(d.table_cells, 1);
  d.poff = L.layout == SD_LAYOUT_PACKED ? c.take<int64_t>(N) : nullptr;
  d.H = c.take<int64_t>(tc);
  d.V = c.take<int64_t>(tc * 6);
  d.S1 = c.take<int64_t>(tc);
  d.S2 = c.take<int64_t>(tc);
  d.Bv = c.take<int64_t>(tc);
  d.Ihat = c.take<int64_t>(ring);
  d.IL = c.take<int64_t>(ring);
  d.Q = c.take<int64_t>(ring * 6);
  d.WB = c.take<int64_t>(ring);
  d.Af = c.take<int64_t>(ring * SD_AN);
  d.Xc = c.take<int64_t>((size_t)N * 4 * SD_XSPAN * wclass);
  d.Yr = c.take<int64_t>((size_t)N * 4 * SD_XSPAN * wclass);
  d.KR = c.take<int64_t>((size_t)SD_KRING * (n + 1) * wclass * wclass * SD_KM);
  d.GL = c.take<int64_t>((size_t)(n + 1) * SD_GAPW * wclass * wclass);
  d.GR = c.take<int64_t>((size_t)(n + 1) * SD_GAPW * wclass * wclass);
  d.cand_cnt = c.take<int32_t>(N);
  d.cand_off = c.take<int64_t>(N);
  d.cand_cap = L.caps.empty() ? nullptr : c.take<int32_t>(N);
  d.cand_c = c.take<int32_t>(std::max<int64_t>(cap, 1));
  d.cand_B = c.take<int64_t>(std::max<int64_t>(cap, 1));
  d.Ext = c.take<int64_t>(N);
  d.mrna = c.take<char>(n + 1);
  d.structure = c.take<char>(n + 1);
  d.tb = c.take<int64_t>(4);
  d.tb_cap = (int)(2 * n + 64);
  d.tb_stack = c.take<int32_t>((size_t)4 * d.tb_cap);
  return c.off;
}

int upload(const sd_energy *E, const HostLattice &L, const SdDesign &d) {
  const int64_t n = L.n, N = L.N;
  std::vector<int32_t> hp(n + 1, 0);
  for (int64_t Lh = 3; Lh <= n; Lh++)
    hp[Lh] = Lh <= 30 ? E->hairpin[Lh]
                      : E->hairpin[30] + (int32_t)(E->lxc * std::log((double)Lh / 30.0));
  std::vector<int64_t> off(N);
  int64_t acc = 0;
  for (int v = 0; v < N; v++) {
    off[v] = acc;
    acc += room(L, v);
  }
  std::vector<int32_t> rooms(N);
  for (int v = 0; v < N; v++) rooms[v] = room(L, v);
  std::vector<SdFlatEdge> fo(std::max(L.E, 1)), fi(std::max(L.E, 1));
  std::vector<int32_t> fo_off(N + 1), fi_off(N + 1);
  sd_internal_flatten((int)N, L.out.data(), L.out_cnt.data(), L.in.data(), L.in_cnt.data(), L.maxin,
                      fo.data(), fo_off.data(), fi.data(), fi_off.data());
  auto cp = [](const void *dst, const void *src, size_t bytes) {
    return bytes == 0 || cudaMemcpy(const_cast<void *>(dst), src, bytes, cudaMemcpyHostToDevice) ==
                             cudaSuccess;
  };
  bool ok = cp(d.lstart, L.lstart.data(), (n + 2) * 4) && cp(d.layer, L.layer.data(), N * 4) &&
            cp(d.out, L.out.data(), L.out.size() * sizeof(SdEdge)) &&
            cp(d.out_cnt, L.out_cnt.data(), N) &&
            cp(d.in, L.in.data(), L.in.size() * sizeof(SdEdge)) && cp(d.in_cnt, L.in_cnt.data(), N) &&
            cp(d.in_mask, L.in_mask.data(), N) && cp(d.out_mask, L.out_mask.data(), N) &&
            cp(d.hp_len, hp.data(), (n + 1) * 4) && cp(d.cand_off, off.data(), N * 8) &&
            (!d.cand_cap || cp(d.cand_cap, rooms.data(), N * 4)) &&
            cp(d.fo, fo.data(), (size_t)L.E * sizeof(SdFlatEdge)) &&
            cp(d.fi, fi.data(), (size_t)L.E * sizeof(SdFlatEdge)) &&
            cp(d.fo_off, fo_off.data(), (N + 1) * 4) && cp(d.fi_off, fi_off.data(), (N + 1) * 4);
  if (ok && d.poff) {
    const std::vector<int64_t> po = packed_offsets(L);
    ok = cp(d.poff, po.data(), N * 8);
  }
  return ok ? SD_OK : SD_ECUDA;
}

}  // namespace

namespace {
struct MotifAutomaton;
int plan_create(const sd_energy *energy, const sd_predictor *pred, double margin, int count,
                const char *const *proteins, const double *codon_weights, int weights_shared,
                const double *lambdas, sd_plan **out, int *item_status, int layout = SD_LAYOUT_SPAN,
                const MotifAutomaton *motifs = nullptr);
}

namespace {
// motif list -> automaton; SD_EINVAL for an empty or non-ACGU motif, more
// than 64 motifs or a motif longer than 32 nucleotides
int motif_automaton(const char *const *motifs, int nmotifs, MotifAutomaton &M) {
  if (nmotifs < 0 || nmotifs > 64 || (nmotifs > 0 && !motifs)) return SD_EINVAL;
  std::vector<std::string> v;
  for (int k = 0; k < nmotifs; k++) {
    if (!motifs[k]) return SD_EINVAL;
    const std::string m = motifs[k];
    if (m.empty() || m.size() > 32 || m.find_first_not_of("ACGU") != std::string::npos)
      return SD_EINVAL;
    v.push_back(m);
  }
  M.build(v);
  return SD_OK;
}
}  // namespace

extern "C" int sd_plan_create_motifs(const sd_energy *energy, int count,
                                     const char *const *proteins, const double *codon_weights,
                                     int weights_shared, const double *lambdas,
                                     const char *const *motifs, int nmotifs, sd_plan **out,
                                     int *item_status) {
  MotifAutomaton M;
  int rc = motif_automaton(motifs, nmotifs, M);
  if (rc != SD_OK) {
    if (out) *out = nullptr;
    return rc;
  }
  return plan_create(energy, nullptr, 0.0, count, proteins, codon_weights, weights_shared, lambdas,
                     out, item_status, SD_LAYOUT_SPAN, &M);
}

extern "C" int sd_design_motifs(const sd_energy *energy, const char *protein,
                                const double *codon_weights, double lambda,
                                const char *const *motifs, int nmotifs, sd_result *out) {
  if (!energy || !protein || !codon_weights || !out) return SD_EINVAL;
  sd_plan *p = nullptr;
  int st = SD_OK;
  int rc = sd_plan_create_motifs(energy, 1, &protein, codon_weights, 1, &lambda, motifs, nmotifs,
                                 &p, &st);
  if (rc != SD_OK) return rc;
  if (st != SD_OK) {
    sd_plan_free(p);
    return st;
  }
  rc = sd_plan_run(p, nullptr);
  if (rc == SD_OK) rc = sd_plan_results(p, out, &st);
  sd_plan_free(p);
  return rc != SD_OK ? rc : st;
}

extern "C" int sd_plan_create_layout(const sd_energy *energy, int count,
                                     const char *const *proteins, const double *codon_weights,
                                     int weights_shared, const double *lambdas, int layout,
                                     sd_plan **out, int *item_status) {
  if (layout != SD_LAYOUT_SPAN && layout != SD_LAYOUT_SQUARE && layout != SD_LAYOUT_PACKED) {
    if (out) *out = nullptr;
    return SD_EINVAL;
  }
  return plan_create(energy, nullptr, 0.0, count, proteins, codon_weights, weights_shared, lambdas,
                     out, item_status, layout);
}

extern "C" int sd_plan_create(const sd_energy *energy, int count, const char *const *proteins,
                              const double *codon_weights, int weights_shared,
                              const double *lambdas, sd_plan **out, int *item_status) {
  return plan_create(energy, nullptr, 0.0, count, proteins, codon_weights, weights_shared, lambdas,
                     out, item_status);
}

extern "C" int sd_plan_create_predicted(const sd_energy *energy, sd_predictor *pred, double margin,
                                        int count, const char *const *proteins,
                                        const double *codon_weights, int weights_shared,
                                        const double *lambdas, sd_plan **out, int *item_status) {
  if (!pred || !(margin > 0.0)) return SD_EINVAL;
  return plan_create(energy, pred, margin, count, proteins, codon_weights, weights_shared, lambdas,
                     out, item_status);
}

namespace {
// Room of every candidate list from the predictor: the predicted retained
// candidates of codon k (summed over span bands) times `margin`, plus a few,
// for every state whose layer lies in codon k (never above the worst case).
int presize(sd_predictor *pred, double margin, std::vector<PlanItem> &items) {
  std::vector<int> idx;
  int Lmax = 1;
  for (size_t k = 0; k < items.size(); k++)
    if (items[k].status == SD_OK && !items[k].protein.empty()) {
      idx.push_back((int)k);
      Lmax = std::max(Lmax, (int)items[k].protein.size());
    }
  if (idx.empty()) return SD_OK;
  const int B = (int)idx.size();
  std::vector<float> feats((size_t)B * Lmax * SD_PRED_FEATURES, 0.f), y((size_t)B * Lmax * 8);
  std::vector<int> lens(B);
  for (int b = 0; b < B; b++) {
    const PlanItem &it = items[idx[b]];
    lens[b] = (int)it.protein.size();
    int rc = sd_pred_features(it.protein.c_str(), it.w, it.lambda,
                              feats.data() + (size_t)b * Lmax * SD_PRED_FEATURES);
    if (rc != SD_OK) return rc;
  }
  int rc = sd_pred_forward(pred, B, Lmax, feats.data(), lens.data(), y.data());
  if (rc != SD_OK) return rc;
  for (int b = 0; b < B; b++) {
    HostLattice &L = items[idx[b]].L;
    const int A = lens[b];
    std::vector<double> total(A, 0.0);
    for (int k = 0; k < A; k++)
      for (int s = 0; s < 8; s++)
        total[k] += std::expm1(std::max(0.f, y[((size_t)b * Lmax + k) * 8 + s]));
    // predicted S2-scan visits: a candidate c of a list ending at codon k
    // in span band s is visited once per start state before it, about
    // 3k - (typical span of band s) layers
    double visits = 0.0;
    for (int k = 0; k < A; k++)
      for (int s = 0; s < 8; s++) {
        const double span = s == 7 ? 768.0 : 6.0 * std::ldexp(1.0, s);
        visits += std::expm1(std::max(0.f, y[((size_t)b * Lmax + k) * 8 + s])) *
                  std::max(0.0, 3.0 * k - span);
      }
    items[idx[b]].pred_visits = visits;
    L.caps.assign(L.N, 0);
    for (int v = 0; v < L.N; v++) {
      if (L.layer[v] < 1) continue;
      const int k = std::min(A - 1, (L.layer[v] - 1) / 3);
      const double want = std::ceil(margin * total[k]) + 8.0;
      L.caps[v] = (int32_t)std::min<double>(want, worst_room(L, v));
    }
  }
  return SD_OK;
}

int plan_create(const sd_energy *energy, const sd_predictor *cpred, double margin, int count,
                const char *const *proteins, const double *codon_weights, int weights_shared,
                const double *lambdas, sd_plan **out, int *item_status, int layout,
                const MotifAutomaton *motifs) {
  sd_predictor *pred = const_cast<sd_predictor *>(cpred);
  if (!out) return SD_EINVAL;
  *out = nullptr;
  if (!energy || count < 0 || (count > 0 && (!proteins || !codon_weights || !lambdas)))
    return SD_EINVAL;
  if (!sd_internal_on_energy_device(energy)) return SD_EINVAL;
  sd_plan *p = new (std::nothrow) sd_plan();
  if (!p) return SD_ENOMEM;
  p->energy = energy;
  p->items.resize(count);
  size_t total = 0;
  for (int k = 0; k < count; k++) {
    PlanItem &it = p->items[k];
    const double *w = codon_weights + (weights_shared ? 0 : (size_t)64 * k);
    std::memcpy(it.w, w, sizeof(it.w));
    it.lambda = lambdas[k];
    if (!proteins[k] || !(std::isfinite(it.lambda) && it.lambda >= 0.0)) {
      it.status = SD_EINVAL;
      continue;
    }
    it.protein = proteins[k];
    it.L.layout = layout;
    it.status = build_lattice(proteins[k], w, it.lambda, it.L, motifs);
    if (it.status == SD_OK && it.L.n > SD_MAX_NT) it.status = SD_EINVAL;
    if (it.status == SD_OK) it.status = range_check(energy, it.L);
  }
  // the kernel instance: wide when some lattice has layers of more than
  // SD_W states or states with more than SD_MAXIN in-edges; wide plans keep
  // the full tables forward-packed
  for (const auto &it : p->items)
    if (it.status == SD_OK && (it.L.width > SD_W || it.L.maxin > SD_MAXIN)) p->wclass = SD_W_WIDE;
  if (p->wclass != SD_W)
    for (auto &it : p->items) it.L.layout = SD_LAYOUT_PACKED;
  if (pred) {
    int rc = presize(pred, margin, p->items);
    if (rc != SD_OK) {
      delete p;
      return rc;
    }
  }
  for (auto &it : p->items) {
    if (it.status != SD_OK) continue;
    SdDesign d{};
    total += carve(nullptr, it.L, d, p->wclass);
    p->max_n = std::max(p->max_n, it.L.n);
  }
  if (item_status)
    for (int k = 0; k < count; k++) item_status[k] = p->items[k].status;
  // device order: longest design first (the span work queue relies on the
  // designs still running at span g being a prefix of this order)
  {
    std::vector<int> order;
    for (int k = 0; k < count; k++)
      if (p->items[k].status == SD_OK) order.push_back(k);
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return p->items[x].L.n > p->items[y].L.n; });
    p->hdesigns.resize(order.size());
    p->ns.resize(order.size());
    std::vector<int32_t> cpre(order.size() + 1, 0);
    for (size_t r = 0; r < order.size(); r++) {
      p->items[order[r]].dev_index = (int)r;
      p->ns[r] = p->items[order[r]].L.n;
      cpre[r + 1] = cpre[r] + p->ns[r] + 1;
    }
    p->cpre_host = cpre;
    // default fill group: 8 threads per layer pair when a span holds many
    // layer pairs (a large batch), else 32 (sd_plan_autotune measures)
    p->group = p->wclass != SD_W ? 32 : SD_GROUP_BY_SPAN;
  }
  if (!p->hdesigns.empty()) {
    if (cudaMalloc(&p->arena, total) != cudaSuccess) {
      cudaGetLastError();
      delete p;
      return SD_ENOMEM;
    }
    p->arena_bytes = total;
    size_t off = 0;
    for (auto &it : p->items) {
      if (it.dev_index < 0) continue;
      SdDesign &d = p->hdesigns[it.dev_index];
      off += carve(p->arena + off, it.L, d, p->wclass);
      d.status_slot = it.dev_index;
      it.d = d;
      int rc = upload(energy, it.L, d);
      if (rc != SD_OK) {
        sd_plan_free(p);
        return rc;
      }
    }
    if (cudaMalloc(&p->d_designs, sizeof(SdDesign) * p->hdesigns.size()) != cudaSuccess ||
        cudaMemcpy(p->d_designs, p->hdesigns.data(), sizeof(SdDesign) * p->hdesigns.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMalloc(&p->d_cpre, sizeof(int32_t) * p->cpre_host.size()) != cudaSuccess ||
        cudaMemcpy(p->d_cpre, p->cpre_host.data(), sizeof(int32_t) * p->cpre_host.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
      sd_plan_free(p);
      return SD_ECUDA;
    }
  }
  *out = p;
  return SD_OK;
}
}  // namespace

namespace {
// An event record that is also an event-record node of a graph being captured
// on the stream (a plain record there is only a capture dependency).
void record_timing(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
  else
    cudaEventRecord(ev, st);
}

// Enqueue one whole run on `st`: one launch sequence over all designs, or,
// with a multi-stream schedule, one per bin on the bins' streams, forked
// from and joined back into `st` (the same pattern is captured into graphs).
int enqueue(sd_plan *p, cudaStream_t st, int64_t *nl) {
  void *ev[4] = {p->ev[0], p->ev[1], p->ev[2], p->ev[3]};
  if (p->bins.empty())
    return k_run(p, p->d_designs, (int)p->hdesigns.size(), p->ns.data(), p->d_cpre, st, nl,
                 p->timing ? ev : nullptr);
  if (p->timing) record_timing(p->ev[0], st);
  if (cudaEventRecord(p->fork, st) != cudaSuccess) return -1;
  int64_t total = 0;
  for (auto &b : p->bins) {
    int64_t n1 = 0;
    if (cudaStreamWaitEvent(b.st, p->fork, 0) != cudaSuccess) return -1;
    if (k_run(p, b.d_designs, (int)b.dev.size(), b.ns.data(), b.d_cpre, b.st, &n1, nullptr))
      return -1;
    total += n1;
    if (cudaEventRecord(b.done, b.st) != cudaSuccess ||
        cudaStreamWaitEvent(st, b.done, 0) != cudaSuccess)
      return -1;
  }
  if (p->timing)
    for (int k = 1; k < 4; k++) record_timing(p->ev[k], st);
  *nl = total;
  return 0;
}

// Upload the bins' copies of the design records (after a regrow or a
// change of retention rule touched the plan's records).
int refresh_bins(sd_plan *p) {
  for (auto &b : p->bins) {
    std::vector<SdDesign> h;
    for (int d : b.dev) h.push_back(p->hdesigns[d]);
    if (cudaMemcpy(b.d_designs, h.data(), sizeof(SdDesign) * h.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return SD_ECUDA;
  }
  return SD_OK;
}

void free_bins(sd_plan *p) {
  for (auto &b : p->bins) {
    if (b.d_designs) cudaFree(b.d_designs);
    if (b.d_cpre) cudaFree(b.d_cpre);
    if (b.st) cudaStreamDestroy(b.st);
    if (b.done) cudaEventDestroy(b.done);
  }
  p->bins.clear();
}
}  // namespace

extern "C" int sd_plan_run(sd_plan *p, void *stream) {
  if (!p) return SD_EINVAL;
  p->last_stream = (cudaStream_t)stream;
  if (p->hdesigns.empty()) return SD_OK;
  int64_t nl = 0;
  if (p->use_graph) {
    if (p->gexec && p->graph_timed != p->timing) {
      cudaGraphExecDestroy(p->gexec);
      p->gexec = nullptr;
    }
    if (!p->gexec) {
      if (!p->cap_stream &&
          cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return SD_ECUDA;
      cudaGraph_t graph = nullptr;
      if (cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return SD_ECUDA;
      int rc = enqueue(p, p->cap_stream, &nl);
      cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &graph);
      if (rc != 0 || ce != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return SD_ECUDA;
      }
      ce = cudaGraphInstantiate(&p->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) {
        p->gexec = nullptr;
        return SD_ECUDA;
      }
      p->graph_timed = p->timing;
      p->graph_launches = nl;
    }
    p->launches = p->graph_launches;
    p->timed_run = p->timing;
    return cudaGraphLaunch(p->gexec, (cudaStream_t)stream) == cudaSuccess ? SD_OK : SD_ECUDA;
  }
  int rc = enqueue(p, (cudaStream_t)stream, &nl);
  p->launches = nl;
  p->timed_run = p->timing;
  return rc == 0 ? SD_OK : SD_ECUDA;
}

// Predicted fill work of one design in candidate-visit units: the closed and
// two-loop cells cost about the same per layer pair (a few hundred min-plus
// terms, kLayerPairWork), the multiloop splits one visit per retained
// candidate and start state (predicted by the retention predictor when the
// plan has one, else taken as zero).
static double design_work(const PlanItem &it) {
  constexpr double kLayerPairWork = 300.0;
  const double n = it.L.n;
  return kLayerPairWork * n * (n + 1) / 2 + std::max(0.0, it.pred_visits);
}

extern "C" int sd_plan_set_streams(sd_plan *p, int k) {
  if (!p || k < 1 || k > 16) return SD_EINVAL;
  if (cudaStreamSynchronize(p->last_stream) != cudaSuccess) return SD_ECUDA;
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  free_bins(p);
  const int nd = (int)p->hdesigns.size();
  if (k == 1 || nd < 2) return SD_OK;
  k = std::min(k, nd);
  // longest processing time first: heaviest design to the lightest bin
  std::vector<int> item_of(nd, -1);
  for (size_t q = 0; q < p->items.size(); q++)
    if (p->items[q].dev_index >= 0) item_of[p->items[q].dev_index] = (int)q;
  std::vector<int> order(nd);
  std::vector<double> w(nd);
  for (int d = 0; d < nd; d++) {
    order[d] = d;
    w[d] = design_work(p->items[item_of[d]]);
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return w[x] > w[y]; });
  std::vector<double> load(k, 0.0);
  p->bins.resize(k);
  for (int d : order) {
    const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[b] += w[d];
    p->bins[b].dev.push_back(d);
  }
  int rc = SD_OK;
  if (!p->fork && cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) != cudaSuccess)
    rc = SD_ECUDA;
  for (auto &b : p->bins) {
    if (rc != SD_OK) break;
    // the span work queue needs each bin's designs longest first
    std::stable_sort(b.dev.begin(), b.dev.end(),
                     [&](int x, int y) { return p->ns[x] > p->ns[y]; });
    b.cpre.assign(1, 0);
    for (int d : b.dev) {
      b.ns.push_back(p->ns[d]);
      b.cpre.push_back(b.cpre.back() + p->ns[d] + 1);
    }
    if (cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&b.d_designs, sizeof(SdDesign) * b.dev.size()) != cudaSuccess ||
        cudaMalloc(&b.d_cpre, sizeof(int32_t) * b.cpre.size()) != cudaSuccess ||
        cudaMemcpy(b.d_cpre, b.cpre.data(), sizeof(int32_t) * b.cpre.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
      rc = SD_ECUDA;
  }
  if (rc == SD_OK) rc = refresh_bins(p);
  if (rc != SD_OK) {
    cudaGetLastError();
    free_bins(p);
  }
  return rc;
}

extern "C" int sd_plan_get_streams(const sd_plan *p) {
  return p ? std::max<int>(1, (int)p->bins.size()) : SD_EINVAL;
}

extern "C" int sd_plan_set_graph(sd_plan *p, int enable) {
  if (!p) return SD_EINVAL;
  if (!enable && p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  p->use_graph = enable != 0;
  return SD_OK;
}

extern "C" int sd_plan_count_ops(sd_plan *p, int64_t *ops) {
  if (!p || (!ops && !p->items.empty())) return SD_EINVAL;
  const int nd = (int)p->hdesigns.size();
  std::vector<unsigned long long> h(nd, 0);
  if (nd > 0) {
    unsigned long long *d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned long long) * nd) != cudaSuccess) return SD_ENOMEM;
    int rc = p->wclass == SD_W
                 ? sd_k_count_ops(p->d_designs, nd, p->ns.data(), p->d_cpre, p->energy->d, d,
                                  nullptr, p->group)
                 : sd_k_count_ops_wide(p->d_designs, nd, p->ns.data(), p->d_cpre, p->energy->d,
                                       d, nullptr, 32);
    bool ok = rc == 0 && cudaMemcpy(h.data(), d, sizeof(unsigned long long) * nd,
                                    cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaFree(d);
    if (!ok) return SD_ECUDA;
  }
  for (size_t k = 0; k < p->items.size(); k++)
    ops[k] = p->items[k].dev_index >= 0 ? (int64_t)h[p->items[k].dev_index] : 0;
  return SD_OK;
}

extern "C" int sd_plan_set_timing(sd_plan *p, int enable);
extern "C" int sd_plan_phase_times(const sd_plan *p, float *ms);

extern "C" int sd_plan_set_group(sd_plan *p, int group) {
  if (!p || !(group == SD_GROUP_BY_SPAN || group == 8 || group == 16 || group == 32))
    return SD_EINVAL;
  if (group != p->group && p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  p->group = group;
  return SD_OK;
}

extern "C" int sd_plan_get_group(const sd_plan *p) { return p ? p->group : SD_EINVAL; }

// Autotuner: run the whole plan once per candidate group size (fill timed with
// events on the legacy default stream) and keep the fastest.
extern "C" int sd_plan_autotune(sd_plan *p, float *ms_out) {
  if (!p) return SD_EINVAL;
  static const int cand[4] = {SD_GROUP_BY_SPAN, 8, 16, 32};
  if (p->hdesigns.empty()) return SD_OK;
  const bool had = p->timing;
  int rc = sd_plan_set_timing(p, 1);
  if (rc != SD_OK) return rc;
  float best = 0.0f;
  int best_g = p->group;
  const int ncand = p->wclass != SD_W ? 1 : 4;  // wide layers: groups of 32 only
  for (int k = 0; k < ncand; k++) {
    p->group = p->wclass != SD_W ? 32 : cand[k];
    rc = sd_plan_run(p, nullptr);
    if (rc != SD_OK) break;
    float ms[3];
    rc = sd_plan_phase_times(p, ms);
    if (rc != SD_OK) break;
    if (ms_out) ms_out[k] = ms[0];
    if (k == 0 || ms[0] < best) {
      best = ms[0];
      best_g = p->group;
    }
  }
  p->group = best_g;
  p->timing = had;
  return rc;
}

extern "C" int sd_plan_set_timing(sd_plan *p, int enable) {
  if (!p) return SD_EINVAL;
  if (enable && !p->ev[0])
    for (int k = 0; k < 4; k++)
      if (cudaEventCreate(&p->ev[k]) != cudaSuccess) return SD_ECUDA;
  p->timing = enable != 0;
  return SD_OK;
}

extern "C" int sd_plan_phase_times(const sd_plan *p, float *ms) {
  if (!p || !ms) return SD_EINVAL;
  if (!p->timed_run || p->hdesigns.empty()) return SD_EINVAL;
  if (cudaEventSynchronize(p->ev[3]) != cudaSuccess) return SD_ECUDA;
  for (int k = 0; k < 3; k++)
    if (cudaEventElapsedTime(&ms[k], p->ev[k], p->ev[k + 1]) != cudaSuccess) return SD_ECUDA;
  return SD_OK;
}

extern "C" int64_t sd_plan_launches(const sd_plan *p) { return p ? p->launches : 0; }
extern "C" int64_t sd_plan_device_bytes(const sd_plan *p) {
  return p ? (int64_t)p->arena_bytes : 0;
}

extern "C" int sd_k_count(const SdDesign *d_designs, int count, int64_t *d_out, void *stream);

// A presized candidate list that overflowed invalidates its design's run.
// The regrow pass gives each such design worst-case room (a buffer of its
// own, kept for later runs of the plan) and repeats the whole path for those
// designs only, as one sub-batch in the plan's device order.
namespace {
int regrow_if_needed(sd_plan *p) {
  std::vector<int> over;  // item indices, in device order
  std::vector<std::pair<int, int>> by_dev;
  for (size_t k = 0; k < p->items.size(); k++) {
    PlanItem &it = p->items[k];
    if (it.status != SD_OK || !it.d.cand_cap) continue;
    int64_t flag = 0;
    if (cudaMemcpy(&flag, it.d.tb + 3, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return SD_ECUDA;
    if (flag & SD_TB_OVERFLOW) by_dev.push_back({it.dev_index, (int)k});
  }
  if (by_dev.empty()) return SD_OK;
  std::sort(by_dev.begin(), by_dev.end());
  for (auto &pr : by_dev) over.push_back(pr.second);
  std::vector<SdDesign> sub;
  std::vector<int> ns;
  std::vector<int32_t> cpre(1, 0);
  for (int k : over) {
    PlanItem &it = p->items[k];
    it.L.caps.clear();
    const int N = it.L.N;
    int64_t cap = 0;
    std::vector<int64_t> off(N);
    for (int v = 0; v < N; v++) {
      off[v] = cap;
      cap += worst_room(it.L, v);
    }
    const size_t off_bytes = ((size_t)N * 8 + 255) & ~(size_t)255;
    const size_t b_bytes = ((size_t)std::max<int64_t>(cap, 1) * 8 + 255) & ~(size_t)255;
    const size_t bytes = off_bytes + b_bytes + (size_t)std::max<int64_t>(cap, 1) * 4;
    char *buf = nullptr;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) return SD_ENOMEM;
    if (it.own_cand) cudaFree(it.own_cand);
    it.own_cand = (int32_t *)buf;
    SdDesign &d = it.d;
    d.cand_off = (int64_t *)buf;
    d.cand_B = (int64_t *)(buf + off_bytes);
    d.cand_c = (int32_t *)(buf + off_bytes + b_bytes);
    d.cand_cap = nullptr;
    if (cudaMemcpy((void *)d.cand_off, off.data(), (size_t)N * 8, cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return SD_ECUDA;
    p->hdesigns[it.dev_index] = d;
    it.regrows++;
    sub.push_back(d);
    ns.push_back(it.L.n);
    cpre.push_back(cpre.back() + it.L.n + 1);
  }
  if (cudaMemcpy(p->d_designs, p->hdesigns.data(), sizeof(SdDesign) * p->hdesigns.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      refresh_bins(p) != SD_OK)
    return SD_ECUDA;
  SdDesign *d_sub = nullptr;
  int32_t *d_cpre = nullptr;
  bool ok = cudaMalloc(&d_sub, sizeof(SdDesign) * sub.size()) == cudaSuccess &&
            cudaMalloc(&d_cpre, sizeof(int32_t) * cpre.size()) == cudaSuccess &&
            cudaMemcpy(d_sub, sub.data(), sizeof(SdDesign) * sub.size(), cudaMemcpyHostToDevice) ==
                cudaSuccess &&
            cudaMemcpy(d_cpre, cpre.data(), sizeof(int32_t) * cpre.size(),
                       cudaMemcpyHostToDevice) == cudaSuccess;
  int64_t nl = 0;
  ok = ok && k_run(p, d_sub, (int)sub.size(), ns.data(), d_cpre, p->last_stream, &nl, nullptr) == 0;
  ok = ok && cudaStreamSynchronize(p->last_stream) == cudaSuccess;
  cudaFree(d_sub);
  cudaFree(d_cpre);
  return ok ? SD_OK : SD_ECUDA;
}
}  // namespace

extern "C" int sd_plan_results(sd_plan *p, sd_result *outs, int *status) {
  if (!p || (!outs && !p->items.empty())) return SD_EINVAL;
  if (cudaStreamSynchronize(p->last_stream) != cudaSuccess) return SD_ECUDA;
  {
    int rc = regrow_if_needed(p);
    if (rc != SD_OK) return rc;
  }
  const int nd = (int)p->hdesigns.size();
  std::vector<int64_t> counts((size_t)nd * 4, 0);
  if (nd > 0) {
    int64_t *d_counts = nullptr;
    if (cudaMalloc(&d_counts, counts.size() * 8) != cudaSuccess) return SD_ENOMEM;
    int rc = p->wclass == SD_W ? sd_k_count(p->d_designs, nd, d_counts, nullptr)
                               : sd_k_count_wide(p->d_designs, nd, d_counts, nullptr);
    bool ok = rc == 0 && cudaMemcpy(counts.data(), d_counts, counts.size() * 8,
                                    cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaFree(d_counts);
    if (!ok) return SD_ECUDA;
  }
  for (size_t k = 0; k < p->items.size(); k++) {
    PlanItem &it = p->items[k];
    sd_result &r = outs[k];
    std::memset(&r, 0, sizeof(r));
    int st = it.status;
    if (st == SD_OK) {
      const SdDesign &d = it.d;
      const int n = it.L.n;
      r.mrna = (char *)std::malloc(n + 1);
      r.structure = (char *)std::malloc(n + 1);
      int64_t tb[4], ext0 = 0;
      if (!r.mrna || !r.structure) {
        st = SD_ENOMEM;
      } else if (cudaMemcpy(r.mrna, d.mrna, n + 1, cudaMemcpyDeviceToHost) != cudaSuccess ||
                 cudaMemcpy(r.structure, d.structure, n + 1, cudaMemcpyDeviceToHost) !=
                     cudaSuccess ||
                 cudaMemcpy(tb, d.tb, sizeof(tb), cudaMemcpyDeviceToHost) != cudaSuccess ||
                 cudaMemcpy(&ext0, d.Ext, 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
        st = SD_ECUDA;
      } else {
        r.mrna[n] = 0;
        r.structure[n] = 0;
        r.n = n;
        r.energy = (int32_t)tb[0];
        r.objective_fx = ext0;
        if (tb[3] & SD_TB_WAIT) st = SD_ETIMEOUT;  // a fill wait gave up
        else if (ext0 >= SD_FINLIM) st = SD_EINFEASIBLE;
        else if (tb[2] != 0 || tb[0] * 4294967296LL + tb[1] != ext0) st = SD_EINTERNAL;
        // FP64 objective from the emitted codons, in codon order
        double cc = 0.0;
        for (int c = 0; st == SD_OK && c + 2 < n; c += 3) {
          int x = nt_code(r.mrna[c]), y = nt_code(r.mrna[c + 1]), z = nt_code(r.mrna[c + 2]);
          if (x < 0 || y < 0 || z < 0) {
            st = SD_EINTERNAL;
            break;
          }
          cc += -std::log(it.w[16 * x + 4 * y + z]);
        }
        r.codon_cost = cc;
        r.objective = (double)r.energy + (100.0 * it.lambda) * cc;
        const int64_t *c4 = &counts[(size_t)it.dev_index * 4];
        r.Z = c4[0];
        r.finite_direct = c4[1];
        r.retained_cells = c4[2];
        r.states = it.L.N;
        r.edges = it.L.E;
        r.regrows = it.regrows;
      }
    }
    if (status) status[k] = st;
  }
  return SD_OK;
}

extern "C" int sd_plan_retention(const sd_plan *p, int item, int32_t *counts) {
  if (!p || !counts || item < 0 || item >= (int)p->items.size()) return SD_EINVAL;
  const PlanItem &it = p->items[item];
  if (it.status != SD_OK) return it.status;
  const int A = it.L.n / 3;
  if (A == 0) return SD_OK;
  if (cudaStreamSynchronize(p->last_stream) != cudaSuccess) return SD_ECUDA;
  int32_t *d = nullptr;
  if (cudaMalloc(&d, sizeof(int32_t) * 8 * A) != cudaSuccess) return SD_ENOMEM;
  int rc = p->wclass == SD_W ? sd_k_retention(p->d_designs, it.dev_index, d, A, nullptr)
                             : sd_k_retention_wide(p->d_designs, it.dev_index, d, A, nullptr);
  bool ok = rc == 0 && cudaMemcpy(counts, d, sizeof(int32_t) * 8 * A, cudaMemcpyDeviceToHost) ==
                           cudaSuccess;
  cudaFree(d);
  return ok ? SD_OK : SD_ECUDA;
}

extern "C" int64_t sd_plan_candidate_room(const sd_plan *p) {
  if (!p) return 0;
  int64_t total = 0;
  for (const auto &it : p->items)
    if (it.status == SD_OK)
      for (int v = 0; v < it.L.N; v++) total += room(it.L, v);
  return total;
}

extern "C" int sd_plan_set_dense(sd_plan *p, int enable) {
  if (!p) return SD_EINVAL;
  for (auto &d : p->hdesigns) d.dense = enable ? 1 : 0;
  for (auto &it : p->items)
    if (it.status == SD_OK) it.d.dense = enable ? 1 : 0;
  if (!p->hdesigns.empty() &&
      cudaMemcpy(p->d_designs, p->hdesigns.data(), sizeof(SdDesign) * p->hdesigns.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return SD_ECUDA;
  return refresh_bins(p);
}

extern "C" int64_t sd_plan_candidate_room_worst(const sd_plan *p) {
  if (!p) return 0;
  int64_t total = 0;
  for (const auto &it : p->items)
    if (it.status == SD_OK)
      for (int v = 0; v < it.L.N; v++) total += worst_room(it.L, v);
  return total;
}

extern "C" int sd_plan_item_size(const sd_plan *p, int item, int32_t *n, int32_t *N, int32_t *E) {
  if (!p || item < 0 || item >= (int)p->items.size()) return SD_EINVAL;
  const PlanItem &it = p->items[item];
  if (n) *n = it.L.n;
  if (N) *N = it.L.N;
  if (E) *E = it.L.E;
  return it.status;
}

extern "C" int sd_plan_edges(const sd_plan *p, int item, int32_t *from, int32_t *to,
                             int32_t *label, int64_t *cost) {
  if (!p || item < 0 || item >= (int)p->items.size()) return SD_EINVAL;
  const HostLattice &L = p->items[item].L;
  for (int e = 0; e < L.E; e++) {
    if (from) from[e] = L.e_from[e];
    if (to) to[e] = L.e_to[e];
    if (label) label[e] = L.e_label[e];
    if (cost) cost[e] = L.e_cost[e];
  }
  return SD_OK;
}

extern "C" int sd_plan_dump(const sd_plan *p, int item, int32_t *layer, int64_t *H, int64_t *V,
                            int64_t *B, int64_t *S1, int64_t *S2, int64_t *Ext, uint8_t *cand) {
  if (!p || item < 0 || item >= (int)p->items.size()) return SD_EINVAL;
  const PlanItem &it = p->items[item];
  if (it.status != SD_OK) return it.status;
  if (cudaDeviceSynchronize() != cudaSuccess) return SD_ECUDA;
  const HostLattice &L = it.L;
  const SdDesign &d = it.d;
  const int64_t N = L.N, NN = N * N;
  const int64_t slots = d.table_cells;
  const std::vector<int64_t> po = L.layout == SD_LAYOUT_PACKED ? packed_offsets(L)
                                                                : std::vector<int64_t>();
  auto fetch = [](std::vector<int64_t> &v, const int64_t *src, int64_t count) {
    v.resize(count);
    return count == 0 ||
           cudaMemcpy(v.data(), src, count * 8, cudaMemcpyDeviceToHost) == cudaSuccess;
  };
  std::vector<int64_t> h, vv, b, s1, s2, ext;
  if ((H && !fetch(h, d.H, slots)) || (V && !fetch(vv, d.V, slots * 6)) ||
      (B && !fetch(b, d.Bv, slots)) || (S1 && !fetch(s1, d.S1, slots)) ||
      (S2 && !fetch(s2, d.S2, slots)) || (Ext && !fetch(ext, d.Ext, N)))
    return SD_ECUDA;
  auto cv = [](int64_t x) { return x >= SD_FINLIM ? (int64_t)SD_EXT_INF : x; };
  if (layer)
    for (int v = 0; v < N; v++) layer[v] = L.layer[v];
  for (int64_t k = 0; k < NN; k++) {
    if (H) H[k] = SD_EXT_INF;
    if (B) B[k] = SD_EXT_INF;
    if (S1) S1[k] = SD_EXT_INF;
    if (S2) S2[k] = SD_EXT_INF;
    if (V)
      for (int t = 0; t < 6; t++) V[k * 6 + t] = SD_EXT_INF;
    if (cand) cand[k] = 0;
  }
  for (int a = 0; a < N; a++)
    for (int bb = L.lstart[L.layer[a] + 1]; bb < N; bb++) {
      const int la = L.layer[a], lb = L.layer[bb];
      const int64_t g = lb - la;
      const int64_t s =
          L.layout == SD_LAYOUT_SQUARE ? (int64_t)a * N + bb
          : L.layout == SD_LAYOUT_PACKED
              ? po[a] + (bb - L.lstart[la + 1])
              : (((g - 1) * (L.n + 1) - (g - 1) * g / 2) + la) * p->wclass * p->wclass +
                    (a - L.lstart[la]) * p->wclass + (bb - L.lstart[lb]);
      const int64_t q = (int64_t)a * N + bb;
      if (H) H[q] = cv(h[s]);
      if (B) B[q] = cv(b[s]);
      if (S1) S1[q] = cv(s1[s]);
      if (S2) S2[q] = cv(s2[s]);
      if (V)
        for (int t = 0; t < 6; t++) V[q * 6 + t] = cv(vv[s * 6 + t]);
    }
  if (Ext)
    for (int v = 0; v < N; v++) Ext[v] = cv(ext[v]);
  if (cand) {
    std::vector<int32_t> cnt(N), cc;
    std::vector<int64_t> off(N);
    if (cudaMemcpy(cnt.data(), d.cand_cnt, N * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(off.data(), d.cand_off, N * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return SD_ECUDA;
    for (int bb = 0; bb < N; bb++) {
      cnt[bb] = std::min(cnt[bb], room(it.L, bb));  // a presized list that overflowed
      cc.resize(std::max(cnt[bb], 1));
      if (cnt[bb] > 0 && cudaMemcpy(cc.data(), d.cand_c + off[bb], (size_t)cnt[bb] * 4,
                                    cudaMemcpyDeviceToHost) != cudaSuccess)
        return SD_ECUDA;
      for (int k = 0; k < cnt[bb]; k++) {
        const int c = it.L.lstart[cc[k] >> SD_CAND_SHIFT] + (cc[k] & ((1 << SD_CAND_SHIFT) - 1));
        cand[(int64_t)c * N + bb] = 1;
      }
    }
  }
  return SD_OK;
}

extern "C" void sd_plan_free(sd_plan *p) {
  if (!p) return;
  if (p->arena) cudaFree(p->arena);
  if (p->d_designs) cudaFree(p->d_designs);
  if (p->d_cpre) cudaFree(p->d_cpre);
  for (auto &it : p->items)
    if (it.own_cand) cudaFree(it.own_cand);
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  free_bins(p);
  if (p->fork) cudaEventDestroy(p->fork);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  for (int k = 0; k < 4; k++)
    if (p->ev[k]) cudaEventDestroy(p->ev[k]);
  delete p;
}

// ---------------------------------------------------------------------------
// one-call conveniences
// ---------------------------------------------------------------------------
extern "C" int sd_design_batch(const sd_energy *energy, int count, const char *const *proteins,
                               const double *codon_weights, int weights_shared,
                               const double *lambdas, sd_result *outs, int *status) {
  if (!energy || count < 0 || (count > 0 && (!outs || !status))) return SD_EINVAL;
  sd_plan *p = nullptr;
  int rc = sd_plan_create(energy, count, proteins, codon_weights, weights_shared, lambdas, &p,
                          status);
  if (rc != SD_OK) return rc;
  rc = sd_plan_run(p, nullptr);
  if (rc == SD_OK) rc = sd_plan_results(p, outs, status);
  sd_plan_free(p);
  return rc;
}

extern "C" int sd_design(const sd_energy *energy, const char *protein, const double *codon_weights,
                         double lambda, sd_result *out) {
  if (!energy || !protein || !codon_weights || !out) return SD_EINVAL;
  int st = SD_OK;
  int rc = sd_design_batch(energy, 1, &protein, codon_weights, 1, &lambda, out, &st);
  return rc != SD_OK ? rc : st;
}

extern "C" void sd_result_free(sd_result *r) {
  if (!r) return;
  std::free(r->mrna);
  std::free(r->structure);
  r->mrna = r->structure = nullptr;
}

extern "C" const char *sd_strerror(int code) {
  switch (code) {
    case SD_OK: return "ok";
    case SD_EINVAL: return "invalid argument";
    case SD_ERANGE: return "objective outside the exact fixed-point range";
    case SD_EINFEASIBLE: return "empty design language";
    case SD_ENOMEM: return "out of memory";
    case SD_ECUDA: return "CUDA runtime error";
    case SD_ETIMEOUT: return "bounded device wait expired";
    case SD_EINTERNAL: return "traceback did not reproduce the DP value";
    case SD_ESIZE: return "design larger than the fixed scratch of sd_design_noalloc";
    default: return "unknown error";
  }
}

// ---------------------------------------------------------------------------
// internal helpers shared with the fixed-scratch entry point (sd_noalloc.cu)
// ---------------------------------------------------------------------------
extern "C" char sd_internal_translate(int x, int y, int z) { return translate(x, y, z); }
extern "C" void sd_internal_flatten(int N, const SdEdge *out, const uint8_t *out_cnt,
                                    const SdEdge *in, const uint8_t *in_cnt, int maxin,
                                    SdFlatEdge *fo,
                                    int32_t *fo_off, SdFlatEdge *fi, int32_t *fi_off) {
  int32_t eo = 0, ei = 0;
  for (int v = 0; v < N; v++) {
    fo_off[v] = eo;
    for (int k = 0; k < out_cnt[v]; k++) {
      const SdEdge &e = out[(size_t)v * SD_MAXOUT + k];
      fo[eo++] = SdFlatEdge{v, e.other * 4 + e.label, e.cost};
    }
    fi_off[v] = ei;
    for (int k = 0; k < in_cnt[v]; k++) {
      const SdEdge &e = in[(size_t)v * maxin + k];
      fi[ei++] = SdFlatEdge{v, e.other * 4 + e.label, e.cost};
    }
  }
  fo_off[N] = eo;
  fi_off[N] = ei;
}
extern "C" int64_t sd_internal_codon_fx(double lambda, double w) { return codon_fx(lambda, w); }
extern "C" int sd_internal_range_check(const sd_energy *E, int n, double qmax_sum) {
  HostLattice L;
  L.n = n;
  L.qmax_sum = qmax_sum;
  return range_check(E, L);
}
extern "C" const SdParams *sd_internal_device_params(const sd_energy *E) { return E ? E->d : nullptr; }
// The energy set's device copy lives on the device that was current when it
// was loaded; kernels launched with another device current would read
// another GPU's memory.
extern "C" int sd_internal_on_energy_device(const sd_energy *E) {
  int dev = -1;
  return E && cudaGetDevice(&dev) == cudaSuccess && dev == E->device;
}
extern "C" int32_t sd_internal_hairpin_len(const sd_energy *E, int L) {
  if (L < 3) return 0;
  return L <= 30 ? E->hairpin[L] : E->hairpin[30] + (int32_t)(E->lxc * std::log((double)L / 30.0));
}

