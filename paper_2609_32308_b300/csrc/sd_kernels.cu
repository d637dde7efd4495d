// sd_kernels.cu -- sm_103a kernels of the exact codon-lattice design DP.
//
// Span wavefront (Algorithm 1, Sec. 5).  One launch per span g processes every
// layer pair (i, i+g) of every design in the batch (grid.y = design).  The
// paper separates closed/gap values, multiloop values and exterior values by
// barriers; here all phases of one layer pair run in the thread that owns it,
// because each of them only reads smaller spans or the same cell:
//   H      min path cost a->b (gap cells)                       span g-1
//   Ihat   inner pair + its loop-side mismatch (two-loop inner)  span g-2
//   IL     generic internal loops below an outer pair            spans g-2..g-26
//   V_t    typed closed value (Sec. 4.1)                         Q at span g-2
//   S2     Eq. (sparse2): edge extension + candidate splits      spans < g
//   S1,B   Eq. (branch), P_S, S1 = min(B, P_S), strict test B < P_S (Eq. candidates)
//   Q_t    hairpin / two-loop / multiloop interior for outer type t (read by V at g+2)
// The owner of layer pair (i, i+g) is the only writer of C_b for b on layer
// i+g at span g (Sec. 5 endpoint ownership), and it scans C_b before it
// appends, so no lock or barrier is needed inside a span.
//
// The exterior (final-column) values and the canonical traceback run after
// the fill, one block per design.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sd_internal.h"

namespace {

__constant__ int c_pair5[6] = {0, 1, 2, 3, 2, 3};
__constant__ int c_pair3[6] = {3, 2, 1, 0, 3, 2};
__constant__ int c_rev[6] = {3, 2, 1, 0, 5, 4};

__device__ __forceinline__ int64_t fx(int e) { return (int64_t)e * 4294967296LL; }
__device__ __forceinline__ int64_t nrm(int64_t v) { return v >= SD_FINLIM ? SD_INF : v; }
__device__ __forceinline__ int64_t mn(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ bool fin(int64_t v) { return v < SD_FINLIM; }

__device__ __forceinline__ int64_t diag_off(int64_t n, int64_t g) {
  return (g - 1) * (n + 1) - (g - 1) * g / 2;
}

struct Lat {
  const SdDesign &D;
  __device__ Lat(const SdDesign &d) : D(d) {}
  __device__ __forceinline__ int layer(int v) const { return __ldg(&D.layer[v]); }
  __device__ __forceinline__ int lstart(int l) const { return __ldg(&D.lstart[l]); }
  __device__ __forceinline__ int64_t slot(int x, int y, int lx, int ly) const {
    return (diag_off(D.n, ly - lx) + lx) * SD_SLOTS + (x - lstart(lx)) * SD_W + (y - lstart(ly));
  }
  __device__ __forceinline__ int64_t rslot(int x, int y, int lx, int ly) const {
    return ((int64_t)((ly - lx) % SD_RING) * (D.n + 1) + lx) * SD_SLOTS + (x - lstart(lx)) * SD_W +
           (y - lstart(ly));
  }
  // min path cost x -> y; 0 for x == y; +inf without a path
  __device__ __forceinline__ int64_t Hp(int x, int y) const {
    if (x == y) return 0;
    int lx = layer(x), ly = layer(y);
    if (ly <= lx) return SD_INF;
    return D.H[slot(x, y, lx, ly)];
  }
  __device__ __forceinline__ int64_t Vt(int c, int d, int t) const {
    int lc = layer(c), ld = layer(d);
    if (ld - lc < 5) return SD_INF;
    return D.V[slot(c, d, lc, ld) * 6 + t];
  }
  __device__ __forceinline__ int64_t S1(int x, int y) const {
    int lx = layer(x), ly = layer(y);
    if (ly <= lx) return SD_INF;
    return D.S1[slot(x, y, lx, ly)];
  }
  __device__ __forceinline__ int64_t S2(int x, int y) const {
    int lx = layer(x), ly = layer(y);
    if (ly <= lx) return SD_INF;
    return D.S2[slot(x, y, lx, ly)];
  }
  __device__ __forceinline__ int64_t Bv(int x, int y) const {
    int lx = layer(x), ly = layer(y);
    if (ly - lx < 5) return SD_INF;
    return D.Bv[slot(x, y, lx, ly)];
  }
  __device__ __forceinline__ int nout(int v) const { return D.out_cnt[v]; }
  __device__ __forceinline__ int nin(int v) const { return D.in_cnt[v]; }
  __device__ __forceinline__ SdEdge out(int v, int k) const { return D.out[v * SD_MAXOUT + k]; }
  __device__ __forceinline__ SdEdge in(int v, int k) const { return D.in[v * SD_MAXIN + k]; }
  __device__ __forceinline__ int out_with_label(int v, int lab) const {
    for (int k = 0; k < nout(v); k++)
      if (D.out[v * SD_MAXOUT + k].label == lab) return k;
    return -1;
  }
};

// ---------------------------------------------------------------------------
// loop energies (integer dcal/mol), Sec. 3 model
// ---------------------------------------------------------------------------

// two-loop energy for every class except the generic one (which the fill
// assembles from Ihat / IL); t outer pair, ti inner pair, xi1 = nt i+1,
// xp1 = nt p-1, xq1 = nt q+1, xj1 = nt j-1
__device__ int twoloop_e(const SdParams &P, int t, int ti, int l1, int l2, int xi1, int xp1,
                         int xq1, int xj1) {
  int s = c_rev[ti];
  if (l1 == 0 && l2 == 0) return P.stack[t][s];
  if (l1 == 0 || l2 == 0) {
    int l = l1 + l2;
    if (l == 1) return P.bulge[1] + P.stack[t][s];
    return P.bulge[l] + P.au[t] + P.au[s];
  }
  if (l1 == 1 && l2 == 1) return P.int11[t][s][xi1 * 4 + xj1];
  if (l1 == 1 && l2 == 2) return P.int21[t][s][xi1 * 16 + xq1 * 4 + xj1];
  if (l1 == 2 && l2 == 1) return P.int21[s][t][xq1 * 16 + xi1 * 4 + xp1];
  if (l1 == 2 && l2 == 2) return P.int22[t][s][xi1 * 64 + xp1 * 16 + xq1 * 4 + xj1];
  int d = l1 > l2 ? l1 - l2 : l2 - l1;
  int asym = min(P.maxninio, P.ninio * d);
  if (l1 == 1 || l2 == 1)
    return P.interior[l1 + l2] + asym + P.mm1n[t][xi1 * 4 + xj1] + P.mm1n[s][xq1 * 4 + xp1];
  if ((l1 == 2 && l2 == 3) || (l1 == 3 && l2 == 2))
    return P.interior[5] + P.ninio + P.mm23[t][xi1 * 4 + xj1] + P.mm23[s][xq1 * 4 + xp1];
  return P.interior[l1 + l2] + asym + P.mmI[t][xi1 * 4 + xj1] + P.mmI[s][xq1 * 4 + xp1];
}

__device__ __forceinline__ int hairpin_generic_e(const SdParams &P, const int32_t *hp_len, int t,
                                                 int L, int f, int l) {
  if (L == 3) return __ldg(&hp_len[3]) + P.au[t];
  return __ldg(&hp_len[L]) + P.mmH[t][f * 4 + l];
}

// hairpin energy of the complete hairpin (pair t, loop labels lab[0..L-1])
__device__ int hairpin_seq_e(const SdParams &P, const int32_t *hp_len, int t, const int *lab,
                             int L) {
  int s = L == 3 ? 0 : L == 4 ? 1 : L == 6 ? 2 : -1;
  if (s >= 0) {
    int code = c_pair5[t];
    for (int k = 0; k < L; k++) code |= lab[k] << (2 * (k + 1));
    code |= c_pair3[t] << (2 * (L + 1));
    for (int k = 0; k < P.nspecial[s]; k++)
      if (P.special_code[s][k] == code) return P.special_e[s][k];
  }
  return hairpin_generic_e(P, hp_len, t, L, lab[0], lab[L - 1]);
}

// Enumerate the interior paths x -> y of L in {3,4,6} edges in lexicographic
// label order.  mode 0: return the min of E + cost.  mode 1: find the first
// path whose E + cost equals target; record its out-edge indices.
__device__ int64_t hairpin_enum(const Lat &G, const SdParams &P, int x, int y, int t, int L,
                                int mode, int64_t target, int *rec_k, int *rec_energy) {
  int st[8], kk[8], lab[8];
  int64_t cs[8];
  int64_t best = SD_INF;
  int depth = 0;
  st[0] = x;
  kk[0] = 0;
  cs[0] = 0;
  while (depth >= 0) {
    if (depth == L) {
      int e = hairpin_seq_e(P, G.D.hp_len, t, lab, L);
      int64_t v = fx(e) + cs[L];
      if (mode == 0) {
        best = mn(best, v);
      } else if (v == target) {
        for (int q = 0; q < L; q++) rec_k[q] = kk[q] - 1;
        *rec_energy = e;
        return v;
      }
      depth--;
      continue;
    }
    int v = st[depth];
    int k = kk[depth]++;
    if (k >= G.nout(v)) {
      depth--;
      continue;
    }
    SdEdge e = G.out(v, k);
    if (depth + 1 == L ? e.other != y : !fin(G.Hp(e.other, y))) continue;
    lab[depth] = e.label;
    st[depth + 1] = e.other;
    cs[depth + 1] = cs[depth] + e.cost;
    kk[depth + 1] = 0;
    depth++;
  }
  return mode == 0 ? best : SD_INF;
}

// ---------------------------------------------------------------------------
// closed-interior value Q_t(x, y): the loop closed by an outer pair of type t
// whose interior path runs from x (after the 5' nucleotide) to y (before the
// 3' nucleotide): hairpin, two-loops (all classes), multiloop.
// ---------------------------------------------------------------------------
// Algorithmic work accounting (counting variant only): every min-plus term
// whose operands are finite adds 2 * (int64 additions + 1 min) INT32 slots.
#define TERM(k) \
  do {                         \
    if (COUNT) ops += 2 * ((k) + 1); \
  } while (0)

template <bool COUNT>
__device__ int64_t q_value(const Lat &G, const SdParams &P, int x, int y, int t, int lx, int ly,
                           unsigned long long &ops) {
  const SdDesign &D = G.D;
  int g = ly - lx;
  int64_t best = SD_INF;
  // hairpin
  if (g >= 3) {
    if (g == 3 || g == 4 || g == 6) {
      best = hairpin_enum(G, P, x, y, t, g, 0, 0, nullptr, nullptr);
      TERM(g);
    } else {
      for (int a = 0; a < G.nout(x); a++) {
        SdEdge e1 = G.out(x, a);
        for (int b = 0; b < G.nin(y); b++) {
          SdEdge e2 = G.in(y, b);
          int64_t h = G.Hp(e1.other, e2.other);
          if (!fin(h)) continue;
          best = mn(best, fx(hairpin_generic_e(P, D.hp_len, t, g, e1.label, e2.label)) + e1.cost +
                              e2.cost + h);
          TERM(3);
        }
      }
    }
  }
  if (g >= 5) {
    // stack and bulges with the inner pair at x (l1 = 0)
    for (int l2 = 0; l2 <= SD_MAXTWO && g - l2 >= 5; l2++) {
      int ld = ly - l2;
      for (int d = G.lstart(ld); d < G.lstart(ld + 1); d++) {
        int64_t h = G.Hp(d, y);
        if (!fin(h)) continue;
        for (int ti = 0; ti < 6; ti++) {
          int64_t v = G.Vt(x, d, ti);
          if (!fin(v)) continue;
          best = mn(best, v + h + fx(twoloop_e(P, t, ti, 0, l2, 0, 0, 0, 0)));
          TERM(2);
        }
      }
    }
    // bulges with the inner pair ending at y (l2 = 0)
    for (int l1 = 1; l1 <= SD_MAXTWO && g - l1 >= 5; l1++) {
      int lc = lx + l1;
      for (int c = G.lstart(lc); c < G.lstart(lc + 1); c++) {
        int64_t h = G.Hp(x, c);
        if (!fin(h)) continue;
        for (int ti = 0; ti < 6; ti++) {
          int64_t v = G.Vt(c, y, ti);
          if (!fin(v)) continue;
          best = mn(best, v + h + fx(twoloop_e(P, t, ti, l1, 0, 0, 0, 0, 0)));
          TERM(2);
        }
      }
    }
    // l1 = 1: 1x1, 1x2, 1xn
    for (int a = 0; a < G.nout(x); a++) {
      SdEdge ec = G.out(x, a);
      int c = ec.other, p = ec.label;
      for (int l2 = 1; l2 <= SD_MAXTWO - 1 && g - 1 - l2 >= 5; l2++) {
        int ld = ly - l2;
        for (int d = G.lstart(ld); d < G.lstart(ld + 1); d++) {
          int64_t vv[6];
          bool any = false;
          for (int ti = 0; ti < 6; ti++) {
            vv[ti] = G.Vt(c, d, ti);
            any |= fin(vv[ti]);
          }
          if (!any) continue;
          if (l2 == 1) {
            for (int b = 0; b < G.nout(d); b++) {
              SdEdge er = G.out(d, b);
              if (er.other != y) continue;
              for (int ti = 0; ti < 6; ti++)
                if (fin(vv[ti]))
                {
                  best = mn(best, vv[ti] + ec.cost + er.cost +
                                      fx(twoloop_e(P, t, ti, 1, 1, p, p, er.label, er.label)));
                  TERM(3);
                }
            }
          } else if (l2 == 2) {
            for (int b = 0; b < G.nout(d); b++) {
              SdEdge r1 = G.out(d, b);
              for (int b2 = 0; b2 < G.nout(r1.other); b2++) {
                SdEdge r2 = G.out(r1.other, b2);
                if (r2.other != y) continue;
                for (int ti = 0; ti < 6; ti++)
                  if (fin(vv[ti]))
                  {
                    best = mn(best, vv[ti] + ec.cost + r1.cost + r2.cost +
                                        fx(twoloop_e(P, t, ti, 1, 2, p, p, r1.label, r2.label)));
                    TERM(4);
                  }
              }
            }
          } else {
            for (int b = 0; b < G.nout(d); b++) {
              SdEdge r1 = G.out(d, b);
              for (int b2 = 0; b2 < G.nin(y); b2++) {
                SdEdge r2 = G.in(y, b2);
                int64_t h = G.Hp(r1.other, r2.other);
                if (!fin(h)) continue;
                for (int ti = 0; ti < 6; ti++)
                  if (fin(vv[ti]))
                  {
                    best = mn(best, vv[ti] + ec.cost + r1.cost + r2.cost + h +
                                        fx(twoloop_e(P, t, ti, 1, l2, p, p, r1.label, r2.label)));
                    TERM(5);
                  }
              }
            }
          }
        }
      }
    }
    // l2 = 1 with l1 >= 2: 2x1, nx1
    for (int b = 0; b < G.nin(y); b++) {
      SdEdge er = G.in(y, b);
      int d = er.other, r = er.label;
      for (int l1 = 2; l1 <= SD_MAXTWO - 1 && g - 1 - l1 >= 5; l1++) {
        int lc = lx + l1;
        for (int c = G.lstart(lc); c < G.lstart(lc + 1); c++) {
          int64_t vv[6];
          bool any = false;
          for (int ti = 0; ti < 6; ti++) {
            vv[ti] = G.Vt(c, d, ti);
            any |= fin(vv[ti]);
          }
          if (!any) continue;
          if (l1 == 2) {
            for (int a = 0; a < G.nout(x); a++) {
              SdEdge p1 = G.out(x, a);
              for (int a2 = 0; a2 < G.nout(p1.other); a2++) {
                SdEdge p2 = G.out(p1.other, a2);
                if (p2.other != c) continue;
                for (int ti = 0; ti < 6; ti++)
                  if (fin(vv[ti]))
                  {
                    best = mn(best, vv[ti] + er.cost + p1.cost + p2.cost +
                                        fx(twoloop_e(P, t, ti, 2, 1, p1.label, p2.label, r, r)));
                    TERM(4);
                  }
              }
            }
          } else {
            for (int a = 0; a < G.nout(x); a++) {
              SdEdge p1 = G.out(x, a);
              for (int a2 = 0; a2 < G.nin(c); a2++) {
                SdEdge p2 = G.in(c, a2);
                int64_t h = G.Hp(p1.other, p2.other);
                if (!fin(h)) continue;
                for (int ti = 0; ti < 6; ti++)
                  if (fin(vv[ti]))
                  {
                    best = mn(best, vv[ti] + er.cost + p1.cost + p2.cost + h +
                                        fx(twoloop_e(P, t, ti, l1, 1, p1.label, p2.label, r, r)));
                    TERM(5);
                  }
              }
            }
          }
        }
      }
    }
    // 2x2, 2x3, 3x2: explicit 2-edge sides, first/last labels on 3-edge sides
    for (int cls = 0; cls < 3; cls++) {
      int l1 = cls == 2 ? 3 : 2, l2 = cls == 1 ? 3 : 2;
      if (g - l1 - l2 < 5) continue;
      int lc = lx + l1, ld = ly - l2;
      for (int c = G.lstart(lc); c < G.lstart(lc + 1); c++)
        for (int d = G.lstart(ld); d < G.lstart(ld + 1); d++) {
          int64_t vv[6];
          bool any = false;
          for (int ti = 0; ti < 6; ti++) {
            vv[ti] = G.Vt(c, d, ti);
            any |= fin(vv[ti]);
          }
          if (!any) continue;
          // left side: first edge from x, last edge into c
          for (int a = 0; a < G.nout(x); a++) {
            SdEdge p1 = G.out(x, a);
            for (int a2 = 0; a2 < G.nin(c); a2++) {
              SdEdge p2 = G.in(c, a2);
              int64_t hl = G.Hp(p1.other, p2.other);
              if (!fin(hl)) continue;
              for (int b = 0; b < G.nout(d); b++) {
                SdEdge r1 = G.out(d, b);
                for (int b2 = 0; b2 < G.nin(y); b2++) {
                  SdEdge r2 = G.in(y, b2);
                  int64_t hr = G.Hp(r1.other, r2.other);
                  if (!fin(hr)) continue;
                  int64_t base = p1.cost + p2.cost + r1.cost + r2.cost + hl + hr;
                  for (int ti = 0; ti < 6; ti++)
                    if (fin(vv[ti]))
                    {
                      best = mn(best, vv[ti] + base +
                                          fx(twoloop_e(P, t, ti, l1, l2, p1.label, p2.label,
                                                       r1.label, r2.label)));
                      TERM(8);
                    }
                }
              }
            }
          }
        }
    }
    // generic internal loops through IL (span g-2 below the mismatch edges);
    // the smallest one (2x4 around a 5-span inner pair) needs g >= 11
    if (g >= 11) {
      for (int a = 0; a < G.nout(x); a++) {
        SdEdge e1 = G.out(x, a);
        for (int b = 0; b < G.nin(y); b++) {
          SdEdge e2 = G.in(y, b);
          int x2 = e1.other, y2 = e2.other;
          int64_t il = D.IL[G.rslot(x2, y2, lx + 1, ly - 1)];
          if (!fin(il)) continue;
          best = mn(best, il + e1.cost + e2.cost + fx(P.mmI[t][e1.label * 4 + e2.label]));
          TERM(3);
        }
      }
    }
  }
  // multiloop closed by the pair
  if (g >= 10) {
    int64_t s2 = D.S2[G.slot(x, y, lx, ly)];
    if (fin(s2)) {
      best = mn(best, s2 + fx(P.mlclosing + P.mlintern + P.au[t]));
      TERM(1);
    }
  }
  return nrm(best);
}

// ---------------------------------------------------------------------------
// the span kernel
// ---------------------------------------------------------------------------
template <bool COUNT>
__global__ void __launch_bounds__(128) k_fill_span(const SdDesign *__restrict__ designs,
                                                   const SdParams *__restrict__ Pp, int g,
                                                   unsigned long long *ops_out) {
  unsigned long long ops = 0;
  const SdDesign &D = designs[blockIdx.y];
  const SdParams &P = *Pp;
  const int n = D.n;
  if (g > n) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n - g) return;
  const int j = i + g;
  Lat G(D);
  const int a0 = G.lstart(i), wa = G.lstart(i + 1) - a0;
  const int b0 = G.lstart(j), wb = G.lstart(j + 1) - b0;
  const int64_t cell = (diag_off(n, g) + i) * SD_SLOTS;
  const int64_t rcell = ((int64_t)(g % SD_RING) * (n + 1) + i) * SD_SLOTS;
  const int64_t mlb = fx(P.mlbase);

  int64_t Bs[SD_SLOTS], PSs[SD_SLOTS];
  for (int sa = 0; sa < wa; sa++)
    for (int sb = 0; sb < wb; sb++) {
      const int a = a0 + sa, b = b0 + sb, s = sa * SD_W + sb;
      // gap cell
      int64_t h = SD_INF;
      for (int k = 0; k < G.nin(b); k++) {
        SdEdge e = G.in(b, k);
        int64_t hp = G.Hp(a, e.other);
        if (fin(hp)) {
          h = mn(h, hp + e.cost);
          TERM(1);
        }
      }
      D.H[cell + s] = nrm(h);
      // Ihat: inner pair (c,d) one nucleotide inside (a,b), its mismatch
      int64_t ih = SD_INF;
      if (g >= 7)
        for (int k1 = 0; k1 < G.nout(a); k1++) {
          SdEdge e1 = G.out(a, k1);
          for (int k2 = 0; k2 < G.nin(b); k2++) {
            SdEdge e2 = G.in(b, k2);
            for (int ti = 0; ti < 6; ti++) {
              int64_t v = G.Vt(e1.other, e2.other, ti);
              if (!fin(v)) continue;
              ih = mn(ih, v + e1.cost + e2.cost + fx(P.mmI[c_rev[ti]][e2.label * 4 + e1.label]));
              TERM(3);
            }
          }
        }
      D.Ihat[rcell + s] = nrm(ih);
      // IL: generic internal loops with l1 = l1'+2, l2 = l2'+2 around (a,b)
      int64_t il = SD_INF;
      if (g >= 9)
        for (int l1p = 0; l1p <= SD_MAXTWO - 4; l1p++)
          for (int l2p = 0; l1p + l2p <= SD_MAXTWO - 4; l2p++) {
            if (l1p + l2p < 2) continue;  // (0,0) 2x2, (0,1)/(1,0) 2x3 / 3x2
            const int lc = i + l1p, ld = j - l2p;
            if (ld - lc < 7) break;
            const int dd = l1p > l2p ? l1p - l2p : l2p - l1p;
            const int64_t e =
                fx(P.interior[l1p + l2p + 4] + min(P.maxninio, P.ninio * dd));
            for (int c = G.lstart(lc); c < G.lstart(lc + 1); c++) {
              int64_t hl = G.Hp(a, c);
              if (!fin(hl)) continue;
              for (int d = G.lstart(ld); d < G.lstart(ld + 1); d++) {
                int64_t hr = G.Hp(d, b);
                if (!fin(hr)) continue;
                int64_t v = D.Ihat[G.rslot(c, d, lc, ld)];
                if (!fin(v)) continue;
                il = mn(il, hl + v + hr + e);
                TERM(3);
              }
            }
          }
      D.IL[rcell + s] = nrm(il);
      // typed closed values and the branch interface, Eq. (branch)
      int64_t B = SD_INF;
      for (int t = 0; t < 6; t++) {
        int64_t v = SD_INF;
        if (g >= 5) {
          int k1 = G.out_with_label(a, c_pair5[t]);
          if (k1 >= 0) {
            SdEdge e1 = G.out(a, k1);
            const int a1 = e1.other;
            for (int k2 = 0; k2 < G.nin(b); k2++) {
              SdEdge e2 = G.in(b, k2);
              if (e2.label != c_pair3[t]) continue;
              int64_t q = D.Q[G.rslot(a1, e2.other, i + 1, j - 1) * 6 + t];
              if (fin(q)) {
                v = mn(v, q + e1.cost + e2.cost);
                TERM(2);
              }
            }
          }
        }
        v = nrm(v);
        D.V[(cell + s) * 6 + t] = v;
        if (fin(v)) {
          B = mn(B, v + fx(P.mlintern + P.au[t]));
          TERM(1);
        }
      }
      B = nrm(B);
      D.Bv[cell + s] = B;
      // Eq. (sparse2)
      int64_t s2 = SD_INF;
      for (int k = 0; k < G.nin(b); k++) {
        SdEdge e = G.in(b, k);
        if (G.layer(e.other) <= i) continue;
        int64_t v = G.S2(a, e.other);
        if (fin(v)) {
          s2 = mn(s2, v + e.cost + mlb);
          TERM(2);
        }
      }
      {
        const int cnt = D.cand_cnt[b];
        const int64_t off = D.cand_off[b];
        for (int k = 0; k < cnt; k++) {
          const int c = D.cand_c[off + k];
          const int lc = G.layer(c);
          if (lc <= i) break;  // entries are in decreasing layer order
          int64_t v = D.S1[G.slot(a, c, i, lc)];
          if (fin(v)) {
            s2 = mn(s2, v + D.cand_B[off + k]);
            TERM(1);
          }
        }
      }
      s2 = nrm(s2);
      D.S2[cell + s] = s2;
      // P_S with S in place of D, Eq. (partitionable)
      int64_t ps = s2;
      for (int k = 0; k < G.nout(a); k++) {
        SdEdge e = G.out(a, k);
        if (G.layer(e.other) >= j) continue;
        int64_t v = G.S1(e.other, b);
        if (fin(v)) {
          ps = mn(ps, v + e.cost + mlb);
          TERM(2);
        }
      }
      for (int k = 0; k < G.nin(b); k++) {
        SdEdge e = G.in(b, k);
        if (G.layer(e.other) <= i) continue;
        int64_t v = G.S1(a, e.other);
        if (fin(v)) {
          ps = mn(ps, v + e.cost + mlb);
          TERM(2);
        }
      }
      ps = nrm(ps);
      D.S1[cell + s] = mn(B, ps);
      Bs[s] = B;
      PSs[s] = ps;
    }
  // candidate appends (Eq. candidates), ascending-layer order is the reverse
  // of the list, so states of one layer are appended in descending id order
  for (int sb = 0; sb < wb; sb++) {
    const int b = b0 + sb;
    int cnt = D.cand_cnt[b];
    const int64_t off = D.cand_off[b];
    for (int sa = wa - 1; sa >= 0; sa--) {
      const int s = sa * SD_W + sb;
      if (Bs[s] < PSs[s]) {
        D.cand_c[off + cnt] = a0 + sa;
        D.cand_B[off + cnt] = Bs[s];
        cnt++;
      }
    }
    D.cand_cnt[b] = cnt;
  }
  // closed-interior values for the pairs two spans up
  for (int sa = 0; sa < wa; sa++)
    for (int sb = 0; sb < wb; sb++) {
      const int x = a0 + sa, y = b0 + sb, s = sa * SD_W + sb;
      const int inm = D.in_mask[x], outm = D.out_mask[y];
      for (int t = 0; t < 6; t++) {
        int64_t q = SD_INF;
        if (((inm >> c_pair5[t]) & 1) && ((outm >> c_pair3[t]) & 1))
          q = q_value<COUNT>(G, P, x, y, t, i, j, ops);
        D.Q[(rcell + s) * 6 + t] = q;
      }
    }
  if (COUNT) atomicAdd(&ops_out[blockIdx.y], ops);
}

// ---------------------------------------------------------------------------
// exterior suffix values (Sec. 5 final-column exterior DP), one block per design
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t block_min(int64_t v, int64_t *sm) {
  for (int o = 16; o > 0; o >>= 1) v = mn(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sm[w] = v;
  __syncthreads();
  int64_t r = SD_INF;
  for (int k = 0; k < (int)(blockDim.x >> 5); k++) r = mn(r, sm[k]);
  return r;
}

__global__ void __launch_bounds__(256) k_exterior(const SdDesign *__restrict__ designs,
                                                  const SdParams *__restrict__ Pp) {
  const SdDesign &D = designs[blockIdx.x];
  const SdParams &P = *Pp;
  __shared__ int64_t sm[32];
  Lat G(D);
  const int n = D.n, N = D.N;
  if (threadIdx.x == 0) D.Ext[N - 1] = 0;
  __syncthreads();
  for (int k = n - 1; k >= 0; k--) {
    for (int a = G.lstart(k); a < G.lstart(k + 1); a++) {
      int64_t best = SD_INF;
      if ((int)threadIdx.x < G.nout(a)) {
        SdEdge e = G.out(a, threadIdx.x);
        int64_t x = D.Ext[e.other];
        if (fin(x)) best = x + e.cost;
      }
      for (int b = G.lstart(k + 1) + threadIdx.x; b < N; b += blockDim.x) {
        const int lb = G.layer(b);
        if (lb - k < 5) continue;
        const int64_t eb = D.Ext[b];
        if (!fin(eb)) continue;
        const int64_t cs = G.slot(a, b, k, lb) * 6;
        for (int t = 0; t < 6; t++) {
          int64_t v = D.V[cs + t];
          if (fin(v)) best = mn(best, v + fx(P.au[t]) + eb);
        }
      }
      best = block_min(best, sm);
      if (threadIdx.x == 0) D.Ext[a] = nrm(best);
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// canonical traceback (one thread per design); the option orders are fixed:
//   exterior : unpaired out-edges by label, then branches by (state b, type t)
//   V_t(a,b) : per last edge (in-edge order): hairpin (special lengths: paths in
//              lexicographic order; else (first,last) label descriptors), then
//              two-loops in (l1+l2, l1, c, d, inner type, left, right
//              descriptor) order, then the multiloop
//   S2       : edge extension (in-edge order), then candidate splits by
//              ascending (layer, state id) of the split state
//   S1       : direct branch, left peel, right peel, S2
//   B        : smallest pair type attaining it
// ---------------------------------------------------------------------------
struct GapDesc {
  int first, last;
  int64_t cost;
  int x1, k1;  // first edge: out-edge k1 of state x1
  int x2, k2;  // second edge of a 2-edge path
};

struct Tb {
  const SdDesign &D;
  const SdParams &P;
  Lat G;
  int64_t energy, pathcost;
  int err;
  int sp;
  __device__ Tb(const SdDesign &d, const SdParams &p) : D(d), P(p), G(d), energy(0), pathcost(0), err(0), sp(0) {}

  __device__ void emit(int from, int label, int64_t cost) {
    const int pos = G.layer(from);
    if (pos < 0 || pos >= D.n || D.mrna[pos] != 0) {
      err = 2;
      return;
    }
    D.mrna[pos] = "ACGU"[label];
    pathcost += cost;
  }
  __device__ void emit_out(int x, int k) {
    SdEdge e = G.out(x, k);
    emit(x, e.label, e.cost);
  }
  __device__ void push(int type, int a, int b, int t) {
    if (sp >= D.tb_cap) {
      err = 3;
      return;
    }
    int32_t *s = D.tb_stack + 4 * sp++;
    s[0] = type;
    s[1] = a;
    s[2] = b;
    s[3] = t;
  }
  __device__ void set_pair(int pi, int pj) {
    if (D.structure[pi] != '.' || D.structure[pj] != '.') err = 4;
    D.structure[pi] = '(';
    D.structure[pj] = ')';
  }
  // canonical min-cost path x -> y
  __device__ void gap(int x, int y) {
    const int ly = G.layer(y);
    while (x != y && !err) {
      const int64_t v = G.Hp(x, y);
      int moved = 0;
      for (int k = 0; k < G.nout(x); k++) {
        SdEdge e = G.out(x, k);
        if (G.layer(e.other) > ly) continue;
        int64_t h = G.Hp(e.other, y);
        if (fin(h) && h + e.cost == v) {
          emit(x, e.label, e.cost);
          x = e.other;
          moved = 1;
          break;
        }
      }
      if (!moved) err = 5;
    }
  }
  __device__ int descs(int x, int y, int len, GapDesc *o) {
    int m = 0;
    if (len == 0) {
      if (x == y) {
        o[m].first = o[m].last = -1;
        o[m].cost = 0;
        o[m].x1 = o[m].k1 = o[m].x2 = o[m].k2 = -1;
        m++;
      }
      return m;
    }
    if (len == 1) {
      for (int k = 0; k < G.nout(x); k++) {
        SdEdge e = G.out(x, k);
        if (e.other != y) continue;
        o[m].first = o[m].last = e.label;
        o[m].cost = e.cost;
        o[m].x1 = x;
        o[m].k1 = k;
        o[m].x2 = o[m].k2 = -1;
        m++;
      }
      return m;
    }
    if (len == 2) {
      for (int k = 0; k < G.nout(x); k++) {
        SdEdge e = G.out(x, k);
        for (int k2 = 0; k2 < G.nout(e.other); k2++) {
          SdEdge e2 = G.out(e.other, k2);
          if (e2.other != y || m >= 16) continue;
          o[m].first = e.label;
          o[m].last = e2.label;
          o[m].cost = e.cost + e2.cost;
          o[m].x1 = x;
          o[m].k1 = k;
          o[m].x2 = e.other;
          o[m].k2 = k2;
          m++;
        }
      }
      return m;
    }
    for (int f = 0; f < 4; f++) {
      int k = G.out_with_label(x, f);
      if (k < 0) continue;
      SdEdge e = G.out(x, k);
      for (int l = 0; l < 4; l++) {
        int64_t best = SD_INF;
        for (int q = 0; q < G.nin(y); q++) {
          SdEdge ei = G.in(y, q);
          if (ei.label != l) continue;
          int64_t h = G.Hp(e.other, ei.other);
          if (fin(h)) best = mn(best, e.cost + h + ei.cost);
        }
        if (fin(best)) {
          o[m].first = f;
          o[m].last = l;
          o[m].cost = best;
          o[m].x1 = x;
          o[m].k1 = k;
          o[m].x2 = o[m].k2 = -1;
          m++;
        }
      }
    }
    return m;
  }
  __device__ void realize(int y, int len, const GapDesc &g) {
    if (len == 0) return;
    if (len == 1) {
      emit_out(g.x1, g.k1);
      return;
    }
    if (len == 2) {
      emit_out(g.x1, g.k1);
      emit_out(g.x2, g.k2);
      return;
    }
    SdEdge e = G.out(g.x1, g.k1);
    for (int q = 0; q < G.nin(y); q++) {
      SdEdge ei = G.in(y, q);
      if (ei.label != g.last) continue;
      int64_t h = G.Hp(e.other, ei.other);
      if (fin(h) && e.cost + h + ei.cost == g.cost) {
        emit(g.x1, e.label, e.cost);
        gap(e.other, ei.other);
        emit(ei.other, ei.label, ei.cost);
        return;
      }
    }
    err = 6;
  }

  __device__ void trace_V(int a, int b, int t) {
    const int64_t v = G.Vt(a, b, t);
    const int kx = G.out_with_label(a, c_pair5[t]);
    if (!fin(v) || kx < 0) {
      err = 7;
      return;
    }
    const SdEdge ex = G.out(a, kx);
    const int a1 = ex.other;
    set_pair(G.layer(a), G.layer(b) - 1);
    GapDesc gl[16], gr[16];
    for (int k = 0; k < G.nin(b); k++) {
      const SdEdge ey = G.in(b, k);
      if (ey.label != c_pair3[t]) continue;
      const int b1 = ey.other;
      const int lx = G.layer(a1), ly = G.layer(b1);
      const int Ln = ly - lx;
      const int64_t base = ex.cost + ey.cost;
      if (Ln >= 3) {
        if (Ln == 3 || Ln == 4 || Ln == 6) {
          int rk[8], re = 0;
          int64_t got = hairpin_enum(G, P, a1, b1, t, Ln, 1, v - base, rk, &re);
          if (got == v - base) {
            emit(a, ex.label, ex.cost);
            int s = a1;
            for (int q = 0; q < Ln; q++) {
              SdEdge e = G.out(s, rk[q]);
              emit(s, e.label, e.cost);
              s = e.other;
            }
            emit(b1, ey.label, ey.cost);
            energy += re;
            return;
          }
        } else {
          int ng = descs(a1, b1, Ln, gl);
          for (int q = 0; q < ng; q++) {
            int e = hairpin_generic_e(P, D.hp_len, t, Ln, gl[q].first, gl[q].last);
            if (base + fx(e) + gl[q].cost == v) {
              emit(a, ex.label, ex.cost);
              realize(b1, Ln, gl[q]);
              emit(b1, ey.label, ey.cost);
              energy += e;
              return;
            }
          }
        }
      }
      for (int l = 0; l <= SD_MAXTWO; l++)
        for (int l1 = 0; l1 <= l; l1++) {
          const int l2 = l - l1;
          const int lc = lx + l1, ld = ly - l2;
          if (ld - lc < 5) continue;
          for (int c = G.lstart(lc); c < G.lstart(lc + 1); c++)
            for (int d = G.lstart(ld); d < G.lstart(ld + 1); d++) {
              const int ngl = descs(a1, c, l1, gl);
              const int ngr = descs(d, b1, l2, gr);
              for (int ti = 0; ti < 6; ti++) {
                const int64_t vi = G.Vt(c, d, ti);
                if (!fin(vi)) continue;
                for (int p = 0; p < ngl; p++)
                  for (int r = 0; r < ngr; r++) {
                    const int e = twoloop_e(P, t, ti, l1, l2, gl[p].first, gl[p].last,
                                            gr[r].first, gr[r].last);
                    if (base + vi + fx(e) + gl[p].cost + gr[r].cost == v) {
                      emit(a, ex.label, ex.cost);
                      realize(c, l1, gl[p]);
                      realize(b1, l2, gr[r]);
                      emit(b1, ey.label, ey.cost);
                      energy += e;
                      push(1, c, d, ti);
                      return;
                    }
                  }
              }
            }
        }
      if (Ln >= 1) {
        const int64_t s2 = G.S2(a1, b1);
        if (fin(s2) && base + fx(P.mlclosing + P.mlintern + P.au[t]) + s2 == v) {
          emit(a, ex.label, ex.cost);
          emit(b1, ey.label, ey.cost);
          energy += P.mlclosing + P.mlintern + P.au[t];
          push(3, a1, b1, 0);
          return;
        }
      }
    }
    err = 8;
  }
  __device__ void trace_B(int a, int b) {
    const int64_t v = G.Bv(a, b);
    for (int t = 0; t < 6; t++) {
      int64_t x = G.Vt(a, b, t);
      if (fin(x) && x + fx(P.mlintern + P.au[t]) == v) {
        energy += P.mlintern + P.au[t];
        trace_V(a, b, t);
        return;
      }
    }
    err = 9;
  }
  __device__ void trace_S2(int a, int b) {
    const int64_t mlb = fx(P.mlbase);
    const int la = G.layer(a);
    while (!err) {
      const int64_t v = G.S2(a, b);
      if (!fin(v)) {
        err = 10;
        return;
      }
      int moved = 0;
      for (int k = 0; k < G.nin(b); k++) {
        SdEdge e = G.in(b, k);
        if (G.layer(e.other) <= la) continue;
        int64_t x = G.S2(a, e.other);
        if (fin(x) && x + e.cost + mlb == v) {
          emit(e.other, e.label, e.cost);
          energy += P.mlbase;
          b = e.other;
          moved = 1;
          break;
        }
      }
      if (moved) continue;
      const int cnt = D.cand_cnt[b];
      const int64_t off = D.cand_off[b];
      for (int k = cnt - 1; k >= 0; k--) {
        const int c = D.cand_c[off + k];
        if (G.layer(c) <= la) continue;
        const int64_t x = G.S1(a, c);
        if (fin(x) && x + D.cand_B[off + k] == v) {
          push(2, a, c, 0);
          push(4, c, b, 0);
          return;
        }
      }
      err = 11;
      return;
    }
  }
  __device__ void trace_S1(int a, int b) {
    const int64_t mlb = fx(P.mlbase);
    while (!err) {
      const int64_t v = G.S1(a, b);
      if (!fin(v)) {
        err = 12;
        return;
      }
      if (G.Bv(a, b) == v) {
        trace_B(a, b);
        return;
      }
      const int la = G.layer(a), lb = G.layer(b);
      int moved = 0;
      for (int k = 0; k < G.nout(a) && !moved; k++) {
        SdEdge e = G.out(a, k);
        if (G.layer(e.other) >= lb) continue;
        int64_t x = G.S1(e.other, b);
        if (fin(x) && x + e.cost + mlb == v) {
          emit(a, e.label, e.cost);
          energy += P.mlbase;
          a = e.other;
          moved = 1;
        }
      }
      if (moved) continue;
      for (int k = 0; k < G.nin(b) && !moved; k++) {
        SdEdge e = G.in(b, k);
        if (G.layer(e.other) <= la) continue;
        int64_t x = G.S1(a, e.other);
        if (fin(x) && x + e.cost + mlb == v) {
          emit(e.other, e.label, e.cost);
          energy += P.mlbase;
          b = e.other;
          moved = 1;
        }
      }
      if (moved) continue;
      if (G.S2(a, b) == v) {
        trace_S2(a, b);
        return;
      }
      err = 13;
      return;
    }
  }
  __device__ void run() {
    const int n = D.n, N = D.N;
    int a = 0;
    const int tstate = N - 1;
    if (!fin(D.Ext[0])) {
      err = 14;
      return;
    }
    while (a != tstate && !err) {
      const int64_t v = D.Ext[a];
      int moved = 0;
      for (int k = 0; k < G.nout(a); k++) {
        SdEdge e = G.out(a, k);
        int64_t x = D.Ext[e.other];
        if (fin(x) && x + e.cost == v) {
          emit(a, e.label, e.cost);
          a = e.other;
          moved = 1;
          break;
        }
      }
      if (moved) continue;
      const int la = G.layer(a);
      for (int b = G.lstart(la + 1); b < N && !moved; b++) {
        const int64_t eb = D.Ext[b];
        if (!fin(eb)) continue;
        for (int t = 0; t < 6 && !moved; t++) {
          int64_t x = G.Vt(a, b, t);
          if (fin(x) && x + fx(P.au[t]) + eb == v) {
            energy += P.au[t];
            push(1, a, b, t);
            a = b;
            moved = 1;
          }
        }
      }
      if (!moved) err = 15;
    }
    while (sp > 0 && !err) {
      const int32_t *s = D.tb_stack + 4 * --sp;
      const int type = s[0], x = s[1], y = s[2], t = s[3];
      if (type == 1) trace_V(x, y, t);
      else if (type == 2) trace_S1(x, y);
      else if (type == 3) trace_S2(x, y);
      else trace_B(x, y);
    }
    for (int k = 0; k < n && !err; k++)
      if (D.mrna[k] == 0) err = 16;
    (void)n;
  }
};

__global__ void k_traceback(const SdDesign *__restrict__ designs, const SdParams *__restrict__ Pp) {
  const SdDesign &D = designs[blockIdx.x];
  for (int k = threadIdx.x; k < D.n; k += blockDim.x) {
    D.mrna[k] = 0;
    D.structure[k] = '.';
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  D.mrna[D.n] = 0;
  D.structure[D.n] = 0;
  Tb tb(D, *Pp);
  tb.run();
  D.tb[0] = tb.energy;
  D.tb[1] = tb.pathcost;
  D.tb[2] = tb.err;
}

__global__ void k_clear_cand(const SdDesign *__restrict__ designs) {
  const SdDesign &D = designs[blockIdx.y];
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < D.N; v += gridDim.x * blockDim.x)
    D.cand_cnt[v] = 0;
}

// per design: [0] Z, [1] finite direct intervals, [2] retained cell updates
__global__ void k_count(const SdDesign *__restrict__ designs, unsigned long long *out) {
  const SdDesign &D = designs[blockIdx.y];
  Lat G(D);
  const int n = D.n;
  unsigned long long z = 0, fd = 0, rc = 0;
  for (int g = 1 + blockIdx.x; g <= n; g += gridDim.x)
    for (int i = threadIdx.x; i + g <= n; i += blockDim.x) {
      const int j = i + g;
      const int wa = G.lstart(i + 1) - G.lstart(i), wb = G.lstart(j + 1) - G.lstart(j);
      const int64_t cell = (diag_off(n, g) + i) * SD_SLOTS;
      for (int sa = 0; sa < wa; sa++)
        for (int sb = 0; sb < wb; sb++) {
          const int64_t s = cell + sa * SD_W + sb;
          fd += fin(D.Bv[s]);
          rc += fin(D.S1[s]) + fin(D.S2[s]);
          for (int t = 0; t < 6; t++) rc += fin(D.V[s * 6 + t]);
        }
    }
  if (blockIdx.x == 0)
    for (int v = threadIdx.x; v < D.N; v += blockDim.x) z += D.cand_cnt[v];
  atomicAdd(&out[blockIdx.y * 4 + 0], z);
  atomicAdd(&out[blockIdx.y * 4 + 1], fd);
  atomicAdd(&out[blockIdx.y * 4 + 2], rc + z);
}

}  // namespace

extern "C" int sd_k_count(const SdDesign *d_designs, int count, int64_t *d_out, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_out, 0, sizeof(int64_t) * 4 * count, st) != cudaSuccess) return -1;
  k_count<<<dim3(64, count), 256, 0, st>>>(d_designs, (unsigned long long *)d_out);
  if (cudaGetLastError() != cudaSuccess) return -1;
  return cudaStreamSynchronize(st) == cudaSuccess ? 0 : -1;
}

// Counting pass: the same fill with algorithmic-work counters (INT32 slots
// per design, see TERM); the result tables are identical to sd_k_run's.
extern "C" int sd_k_count_ops(const SdDesign *d_designs, int count, int max_n,
                              const SdParams *d_params, unsigned long long *d_ops, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (count <= 0) return 0;
  if (cudaMemsetAsync(d_ops, 0, sizeof(unsigned long long) * count, st) != cudaSuccess) return -1;
  k_clear_cand<<<dim3(8, count), 256, 0, st>>>(d_designs);
  for (int g = 1; g <= max_n; g++) {
    const int cells = max_n - g + 1;
    dim3 grid((cells + 127) / 128, count);
    k_fill_span<true><<<grid, 128, 0, st>>>(d_designs, d_params, g, d_ops);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

extern "C" int sd_k_run(const SdDesign *d_designs, int count, int max_n, const SdParams *d_params,
                        void *stream, int64_t *launches, void *const *events) {
  cudaStream_t st = (cudaStream_t)stream;
  int64_t nl = 0;
  if (count <= 0) {
    if (launches) *launches = 0;
    return 0;
  }
  k_clear_cand<<<dim3(8, count), 256, 0, st>>>(d_designs);
  nl++;
  if (events) cudaEventRecord((cudaEvent_t)events[0], st);
  for (int g = 1; g <= max_n; g++) {
    const int cells = max_n - g + 1;
    dim3 grid((cells + 127) / 128, count);
    k_fill_span<false><<<grid, 128, 0, st>>>(d_designs, d_params, g, nullptr);
    nl++;
  }
  if (events) cudaEventRecord((cudaEvent_t)events[1], st);
  k_exterior<<<count, 256, 0, st>>>(d_designs, d_params);
  nl++;
  if (events) cudaEventRecord((cudaEvent_t)events[2], st);
  k_traceback<<<count, 128, 0, st>>>(d_designs, d_params);
  nl++;
  if (events) cudaEventRecord((cudaEvent_t)events[3], st);
  if (launches) *launches = nl;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
