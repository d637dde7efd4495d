// sd_noalloc.cu -- one exact design without any device-memory allocation.
//
// Who needs this: callers that may not call cudaMalloc (or any allocator that
// ends in it, torch's caching allocator included) at the time they want a
// design -- for example code running under a host-side memory budget that
// forbids new device allocations, or a service whose GPU memory is carved up
// in advance by someone else.  sd_design and the plan interface allocate the
// packed tables for every call; sd_design_noalloc instead uses one scratch
// array that the library holds for the life of the process.
//
// The scratch is a file-scope static __device__ array of SD_NOALLOC_SCRATCH
// bytes (64 MiB): every GPU that loads the library keeps it until exit.  It
// fits designs of up to a few hundred nucleotides (the exact limit depends on
// the protein: sd_design_noalloc measures the layout and rejects a design that
// does not fit with SD_ESIZE).  Host code may not use the array's name as a
// device address (in host code it is only a stand-in), so the first call on a
// device, with that device current, asks the runtime for the address with
// cudaGetSymbolAddress and keeps it; make that first call before any stream
// capture.  Every call reuses the same scratch (and one host-side lattice
// buffer), so calls that overlap -- from two host threads, or with work still
// in flight on the device -- race: serialise them.  Leftovers of the previous
// call are harmless: the fill writes every table cell before reading it, and
// the candidate counters, the traceback buffers and the result counters are
// cleared at the start of each call.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "../../include/sd.h"
#include "sd_internal.h"

#define SD_NOALLOC_SCRATCH (64u << 20)

static __device__ __align__(256) unsigned char g_sd_noalloc_scratch[SD_NOALLOC_SCRATCH];

namespace {

constexpr int kMaxDevices = 64;
void *g_scratch[kMaxDevices];  // device address of the scratch, per device

// Fixed-capacity host copy of one codon DFA (no heap use on this path).
constexpr int kMaxCodons = 400;
constexpr int kMaxNt = 3 * kMaxCodons;
constexpr int kMaxStates = 5 * kMaxCodons + 1;
struct FixedLattice {
  int n, N, E;
  double qmax_sum;
  int32_t lstart[kMaxNt + 2];
  int32_t layer[kMaxStates];
  SdEdge out[kMaxStates * SD_MAXOUT];
  SdEdge in[kMaxStates * SD_MAXIN];
  uint8_t out_cnt[kMaxStates], in_cnt[kMaxStates], in_mask[kMaxStates], out_mask[kMaxStates];
  int32_t hp[kMaxNt + 1];
  int64_t cand_off[kMaxStates];
  SdFlatEdge fo[kMaxStates * SD_MAXOUT], fi[kMaxStates * SD_MAXOUT];
  int32_t fo_off[kMaxStates + 1], fi_off[kMaxStates + 1];
};
FixedLattice g_lat;

int nt_index(char c) {
  switch (c) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    case 'U': return 3;
    default: return -1;
  }
}

void add_out(FixedLattice &L, int from, int to, int label, int64_t cost) {
  L.out[from * SD_MAXOUT + L.out_cnt[from]++] = SdEdge{to, label, cost};
  L.out_mask[from] |= 1 << label;
}

// The codon trie of Sec. 3, states numbered layer by layer and by codon
// prefix inside a layer, out-edges by label, in-edges by (label, source).
int build_fixed(const char *protein, const double *w, double lambda, FixedLattice &L) {
  const int A = (int)std::strlen(protein);
  if (A > kMaxCodons) return SD_ESIZE;
  for (int k = 0; k < A; k++)
    if (protein[k] == '*' && k != A - 1) return SD_EINVAL;
  L.n = 3 * A;
  L.N = 0;
  L.E = 0;
  L.qmax_sum = 0.0;
  std::memset(L.out_cnt, 0, sizeof(L.out_cnt));
  std::memset(L.in_cnt, 0, sizeof(L.in_cnt));
  std::memset(L.in_mask, 0, sizeof(L.in_mask));
  std::memset(L.out_mask, 0, sizeof(L.out_mask));
  L.lstart[0] = 0;
  L.layer[L.N++] = 0;
  int boundary = 0;
  for (int k = 0; k < A; k++) {
    bool used[4][4][4] = {};
    int cnt = 0;
    double wmax = 0.0, qmax = 0.0;
    for (int x = 0; x < 4; x++)
      for (int y = 0; y < 4; y++)
        for (int z = 0; z < 4; z++) {
          if (sd_internal_translate(x, y, z) != protein[k]) continue;
          const double ww = w[16 * x + 4 * y + z];
          if (!(ww > 0.0 && ww <= 1.0)) return SD_EINVAL;
          used[x][y][z] = true;
          cnt++;
          wmax = ww > wmax ? ww : wmax;
          const double q = (100.0 * lambda) * -std::log(ww);
          qmax = q > qmax ? q : qmax;
        }
    if (cnt == 0 || wmax != 1.0) return SD_EINVAL;
    L.qmax_sum += qmax;
    int first[4], pre[4][4];
    L.lstart[3 * k + 1] = L.N;
    for (int x = 0; x < 4; x++) {
      bool any = false;
      for (int y = 0; y < 4; y++)
        for (int z = 0; z < 4; z++) any |= used[x][y][z];
      first[x] = any ? L.N : -1;
      if (any) L.layer[L.N++] = 3 * k + 1;
    }
    L.lstart[3 * k + 2] = L.N;
    for (int x = 0; x < 4; x++)
      for (int y = 0; y < 4; y++) {
        bool any = false;
        for (int z = 0; z < 4; z++) any |= used[x][y][z];
        pre[x][y] = any ? L.N : -1;
        if (any) L.layer[L.N++] = 3 * k + 2;
      }
    L.lstart[3 * k + 3] = L.N;
    const int next = L.N;
    L.layer[L.N++] = 3 * k + 3;
    for (int x = 0; x < 4; x++)
      if (first[x] >= 0) {
        add_out(L, boundary, first[x], x, 0);
        L.in[first[x] * SD_MAXIN + L.in_cnt[first[x]]++] = SdEdge{boundary, x, 0};
        L.in_mask[first[x]] |= 1 << x;
        L.E++;
      }
    for (int x = 0; x < 4; x++)
      for (int y = 0; y < 4; y++)
        if (pre[x][y] >= 0) {
          add_out(L, first[x], pre[x][y], y, 0);
          L.in[pre[x][y] * SD_MAXIN + L.in_cnt[pre[x][y]]++] = SdEdge{first[x], y, 0};
          L.in_mask[pre[x][y]] |= 1 << y;
          L.E++;
        }
    // third edges; in-edges of the next boundary ordered by (label, source)
    for (int z = 0; z < 4; z++)
      for (int x = 0; x < 4; x++)
        for (int y = 0; y < 4; y++)
          if (used[x][y][z]) {
            const int64_t c = sd_internal_codon_fx(lambda, w[16 * x + 4 * y + z]);
            if (L.in_cnt[next] >= SD_MAXIN) return SD_EINVAL;
            L.in[next * SD_MAXIN + L.in_cnt[next]++] = SdEdge{pre[x][y], z, c};
            L.in_mask[next] |= 1 << z;
            L.E++;
          }
    for (int x = 0; x < 4; x++)
      for (int y = 0; y < 4; y++)
        for (int z = 0; z < 4; z++)
          if (used[x][y][z]) add_out(L, pre[x][y], next, z, sd_internal_codon_fx(lambda, w[16 * x + 4 * y + z]));
    boundary = next;
  }
  L.lstart[L.n + 1] = L.N;
  // the in-edges of a boundary state were added by label, then by (x, y) of
  // the source prefix; prefix ids increase with (x, y), so they are in order
  for (int l = 0; l <= L.n; l++)
    if (L.lstart[l + 1] - L.lstart[l] > SD_W) return SD_EINVAL;
  int64_t acc = 0;
  for (int v = 0; v < L.N; v++) {
    L.cand_off[v] = acc;
    const int lv = L.layer[v] - 4;
    acc += L.lstart[lv > 0 ? lv : 0];
  }
  return SD_OK;
}

size_t up(size_t x) { return (x + 255) & ~(size_t)255; }

// Lay the design out from `base` (nullptr: measure only); returns the bytes
// used, including the device design record and the result counters.
size_t carve_fixed(char *base, const FixedLattice &L, SdDesign &d, SdDesign **rec,
                   int64_t **counts) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char * {
    char *p = base ? base + off : nullptr;
    off = up(off + bytes);
    return p;
  };
  const int64_t n = L.n, N = L.N, ncell = n * (n + 1) / 2;
  const int64_t cap = L.cand_off[N - 1] + L.lstart[(L.layer[N - 1] - 4) > 0 ? L.layer[N - 1] - 4 : 0];
  const size_t ring = (size_t)SD_RING * (n + 1) * SD_SLOTS;
  *rec = (SdDesign *)take(sizeof(SdDesign));
  *counts = (int64_t *)take(4 * sizeof(int64_t));
  take(2 * sizeof(int32_t));  // prefix sums of the one-design work queue (after counts)
  d.n = (int)n;
  d.N = (int)N;
  d.ncell = ncell;
  d.layout = SD_LAYOUT_SPAN;
  d.table_cells = ncell * SD_SLOTS;
  d.poff = nullptr;
  d.maxin = SD_MAXIN;
  d.status_slot = 0;
  d.lstart = (int32_t *)take((n + 2) * 4);
  d.layer = (int32_t *)take(N * 4);
  d.pos = (int32_t *)take(N * 4);
  d.out = (SdEdge *)take(N * SD_MAXOUT * sizeof(SdEdge));
  d.out_cnt = (uint8_t *)take(N);
  d.in = (SdEdge *)take(N * SD_MAXIN * sizeof(SdEdge));
  d.in_cnt = (uint8_t *)take(N);
  d.in_mask = (uint8_t *)take(N);
  d.out_mask = (uint8_t *)take(N);
  d.hp_len = (int32_t *)take((n + 1) * 4);
  d.fo = (SdFlatEdge *)take((L.E > 0 ? L.E : 1) * sizeof(SdFlatEdge));
  d.fo_off = (int32_t *)take((N + 1) * 4);
  d.fi = (SdFlatEdge *)take((L.E > 0 ? L.E : 1) * sizeof(SdFlatEdge));
  d.fi_off = (int32_t *)take((N + 1) * 4);
  d.H = (int64_t *)take(ncell * SD_SLOTS * 8);
  d.V = (int64_t *)take(ncell * SD_SLOTS * 6 * 8);
  d.S1 = (int64_t *)take(ncell * SD_SLOTS * 8);
  d.S2 = (int64_t *)take(ncell * SD_SLOTS * 8);
  d.Bv = (int64_t *)take(ncell * SD_SLOTS * 8);
  d.Ihat = (int64_t *)take(ring * 8);
  d.IL = (int64_t *)take(ring * 8);
  d.Q = (int64_t *)take(ring * 6 * 8);
  d.WB = (int64_t *)take(ring * 8);
  d.Af = (int64_t *)take(ring * SD_AN * 8);
  d.Xc = (int64_t *)take((size_t)N * 4 * SD_XSPAN * SD_W * 8);
  d.Yr = (int64_t *)take((size_t)N * 4 * SD_XSPAN * SD_W * 8);
  d.KR = (int64_t *)take((size_t)SD_KRING * (n + 1) * SD_SLOTS * SD_KM * 8);
  d.GL = (int64_t *)take((size_t)(n + 1) * SD_GAPW * SD_SLOTS * 8);
  d.GR = (int64_t *)take((size_t)(n + 1) * SD_GAPW * SD_SLOTS * 8);
  d.cand_cnt = (int32_t *)take(N * 4);
  d.cand_off = (int64_t *)take(N * 8);
  d.cand_c = (int32_t *)take((cap > 0 ? cap : 1) * 4);
  d.cand_B = (int64_t *)take((cap > 0 ? cap : 1) * 8);
  d.Ext = (int64_t *)take(N * 8);
  d.mrna = take(n + 1);
  d.structure = take(n + 1);
  d.tb = (int64_t *)take(4 * 8);
  d.tb_cap = (int)(2 * n + 64);
  d.tb_stack = (int32_t *)take((size_t)4 * d.tb_cap * 4);
  return off;
}

bool h2d(void *dst, const void *src, size_t bytes) {
  return bytes == 0 || cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
}
bool d2h(void *dst, const void *src, size_t bytes) {
  return bytes == 0 || cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) == cudaSuccess;
}

}  // namespace

extern "C" int sd_design_noalloc(const sd_energy *energy, const char *protein,
                                 const double *codon_weights, double lambda, sd_result *out) {
  if (!energy || !protein || !codon_weights || !out || !out->mrna || !out->structure)
    return SD_EINVAL;
  if (!(std::isfinite(lambda) && lambda >= 0.0)) return SD_EINVAL;
  if (!sd_internal_on_energy_device(energy)) return SD_EINVAL;
  char *mrna = out->mrna, *structure = out->structure;
  FixedLattice &L = g_lat;
  int rc = build_fixed(protein, codon_weights, lambda, L);
  if (rc != SD_OK) return rc;
  rc = sd_internal_range_check(energy, L.n, L.qmax_sum);
  if (rc != SD_OK) return rc;
  for (int Lh = 0; Lh <= L.n; Lh++) L.hp[Lh] = sd_internal_hairpin_len(energy, Lh);
  sd_internal_flatten(L.N, L.out, L.out_cnt, L.in, L.in_cnt, SD_MAXIN, L.fo, L.fo_off, L.fi,
                      L.fi_off);
  // set-up, once per device, with that device current
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SD_ECUDA;
  if (!g_scratch[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sd_noalloc_scratch) != cudaSuccess || !p) return SD_ECUDA;
    g_scratch[dev] = p;
  }
  SdDesign d{};
  SdDesign *rec = nullptr;
  int64_t *counts = nullptr;
  if (carve_fixed(nullptr, L, d, &rec, &counts) > SD_NOALLOC_SCRATCH) return SD_ESIZE;
  carve_fixed((char *)g_scratch[dev], L, d, &rec, &counts);
  const int64_t n = L.n, N = L.N;
  if (!h2d((void *)d.lstart, L.lstart, (n + 2) * 4) || !h2d((void *)d.layer, L.layer, N * 4) ||
      !h2d((void *)d.out, L.out, N * SD_MAXOUT * sizeof(SdEdge)) ||
      !h2d((void *)d.out_cnt, L.out_cnt, N) ||
      !h2d((void *)d.in, L.in, N * SD_MAXIN * sizeof(SdEdge)) ||
      !h2d((void *)d.in_cnt, L.in_cnt, N) || !h2d((void *)d.in_mask, L.in_mask, N) ||
      !h2d((void *)d.out_mask, L.out_mask, N) || !h2d((void *)d.hp_len, L.hp, (n + 1) * 4) ||
      !h2d((void *)d.cand_off, L.cand_off, N * 8) ||
      !h2d((void *)d.fo, L.fo, L.E * sizeof(SdFlatEdge)) ||
      !h2d((void *)d.fi, L.fi, L.E * sizeof(SdFlatEdge)) ||
      !h2d((void *)d.fo_off, L.fo_off, (N + 1) * 4) ||
      !h2d((void *)d.fi_off, L.fi_off, (N + 1) * 4) || !h2d(rec, &d, sizeof(SdDesign)))
    return SD_ECUDA;
  int64_t launches = 0;
  int32_t *cpre = (int32_t *)((char *)counts + 256);  // the 2-int block carved after counts
  const int32_t cpre_h[2] = {0, (int32_t)n + 1};
  const int ns[1] = {(int)n};
  if (!h2d(cpre, cpre_h, sizeof(cpre_h))) return SD_ECUDA;
  if (sd_k_run(rec, 1, ns, cpre, sd_internal_device_params(energy), nullptr, &launches, nullptr,
               32))
    return SD_ECUDA;
  if (sd_k_count(rec, 1, counts, nullptr)) return SD_ECUDA;
  int64_t tb[4], ext0 = 0, cnt[4];
  if (!d2h(mrna, d.mrna, n + 1) || !d2h(structure, d.structure, n + 1) ||
      !d2h(tb, d.tb, sizeof(tb)) || !d2h(&ext0, d.Ext, 8) || !d2h(cnt, counts, sizeof(cnt)))
    return SD_ECUDA;
  mrna[n] = 0;
  structure[n] = 0;
  if (tb[3] & SD_TB_WAIT) return SD_ETIMEOUT;  // a fill wait gave up
  if (ext0 >= SD_FINLIM) return SD_EINFEASIBLE;
  if (tb[2] != 0 || tb[0] * 4294967296LL + tb[1] != ext0) return SD_EINTERNAL;
  double cc = 0.0;
  for (int c = 0; c + 2 < (int)n; c += 3) {
    const int x = nt_index(mrna[c]), y = nt_index(mrna[c + 1]), z = nt_index(mrna[c + 2]);
    if (x < 0 || y < 0 || z < 0) return SD_EINTERNAL;
    cc += -std::log(codon_weights[16 * x + 4 * y + z]);
  }
  std::memset(out, 0, sizeof(*out));
  out->mrna = mrna;
  out->structure = structure;
  out->n = (int32_t)n;
  out->energy = (int32_t)tb[0];
  out->objective_fx = ext0;
  out->codon_cost = cc;
  out->objective = (double)out->energy + (100.0 * lambda) * cc;
  out->Z = cnt[0];
  out->finite_direct = cnt[1];
  out->retained_cells = cnt[2];
  out->states = N;
  out->edges = L.E;
  out->regrows = 0;
  return SD_OK;
}
