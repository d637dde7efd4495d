// sd_kernels.cu -- sm_103a kernels of the exact codon-lattice design DP.
//
// Span wavefront (Algorithm 1, Sec. 5).  One launch per span g processes every
// layer pair (i, i+g) of every design in the batch (grid.y = design), one warp
// per layer pair.  The paper separates closed/gap values, multiloop values and
// exterior values by barriers; here all phases of one layer pair run in the
// warp that owns it, because each only reads smaller spans or the same cell:
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
// Canonical choices.  Next to every value the fill stores the key of the
// option that attains it: the lexicographic minimum of (value, key), with keys
// ordered like the canonical enumeration (the first attaining option wins a
// tie).  Min-plus composition preserves this, so a stored key is exactly the
// canonical choice and the traceback only follows keys.
//
// The exterior (final-column) values and the traceback run after the fill,
// one block per design.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sd_internal.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t KEY_NONE = 0xffffffffu;

__constant__ int c_pair5[6] = {0, 1, 2, 3, 2, 3};
__constant__ int c_pair3[6] = {3, 2, 1, 0, 3, 2};
__constant__ int c_rev[6] = {3, 2, 1, 0, 5, 4};

__device__ __forceinline__ int64_t fx(int e) { return (int64_t)e * 4294967296LL; }
__device__ __forceinline__ bool fin(int64_t v) { return v < SD_FINLIM; }

__device__ __forceinline__ int64_t diag_off(int64_t n, int64_t g) {
  return (g - 1) * (n + 1) - (g - 1) * g / 2;
}

// lexicographic (value, key) minimum
__device__ __forceinline__ void upd(int64_t &bv, uint32_t &bk, int64_t v, uint32_t k) {
  if (v < bv || (v == bv && k < bk)) {
    bv = v;
    bk = k;
  }
}
__device__ __forceinline__ void warp_lexmin(int64_t &v, uint32_t &k) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int64_t v2 = __shfl_xor_sync(FULL, v, o);
    const uint32_t k2 = __shfl_xor_sync(FULL, k, o);
    upd(v, k, v2, k2);
  }
}
__device__ __forceinline__ void settle(int64_t &v, uint32_t &k) {
  if (!fin(v)) {
    v = SD_INF;
    k = KEY_NONE;
  }
}

// Key layout of closed-interior (Q) and typed closed (V) values:
//   [31:27] index of the last edge into b (V only)
//   [26:25] class: 0 hairpin, 1 two-loop, 2 multiloop
//   two-loop: [24:20] l1+l2, [19:15] l1, [14:13] slot of c, [12:11] slot of d,
//             [10:8] inner type, [7:6] fL, [5:4] lL, [3:2] fR, [1:0] lR
//             (first / last nucleotide of the left and right unpaired sides;
//             for a 1-nt side both are its nucleotide, for none both are 0)
//   hairpin : special lengths: the loop labels, first label most significant;
//             otherwise first*4 + last loop nucleotide
// This order is the canonical enumeration order of the options.
__device__ __forceinline__ uint32_t tl_key(int l1, int l2, int cs, int ds, int ti, int fL, int lL,
                                           int fR, int lR) {
  return (1u << 25) | ((uint32_t)(l1 + l2) << 20) | ((uint32_t)l1 << 15) | ((uint32_t)cs << 13) |
         ((uint32_t)ds << 11) | ((uint32_t)ti << 8) | ((uint32_t)fL << 6) | ((uint32_t)lL << 4) |
         ((uint32_t)fR << 2) | (uint32_t)lR;
}
constexpr uint32_t KEY_ML = 2u << 25;
constexpr uint32_t KEY_QMASK = (1u << 27) - 1;
constexpr uint32_t KEY_SPLIT = 1u << 30;  // S2 candidate split / exterior branch

struct Lat {
  const SdDesign &D;
  __device__ Lat(const SdDesign &d) : D(d) {}
  __device__ __forceinline__ int layer(int v) const { return __ldg(&D.layer[v]); }
  __device__ __forceinline__ int lstart(int l) const { return __ldg(&D.lstart[l]); }
  __device__ __forceinline__ int64_t slot(int x, int y, int lx, int ly) const {
    return (diag_off(D.n, ly - lx) + lx) * SD_SLOTS + (x - lstart(lx)) * SD_W + (y - lstart(ly));
  }
  // min path cost x -> y; 0 for x == y; +inf without a path
  __device__ __forceinline__ int64_t Hp(int x, int y) const {
    if (x == y) return 0;
    const int lx = layer(x), ly = layer(y);
    if (ly <= lx) return SD_INF;
    return D.H[slot(x, y, lx, ly)];
  }
  __device__ __forceinline__ int64_t Vt(int c, int d, int t) const {
    const int lc = layer(c), ld = layer(d);
    if (ld - lc < 5) return SD_INF;
    return D.V[slot(c, d, lc, ld) * 6 + t];
  }
  __device__ __forceinline__ int64_t S1(int x, int y) const {
    const int lx = layer(x), ly = layer(y);
    if (ly <= lx) return SD_INF;
    return D.S1[slot(x, y, lx, ly)];
  }
  __device__ __forceinline__ int64_t S2(int x, int y) const {
    const int lx = layer(x), ly = layer(y);
    if (ly <= lx) return SD_INF;
    return D.S2[slot(x, y, lx, ly)];
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

// two-loop energy; t outer pair, ti inner pair, xi1 = nt i+1, xp1 = nt p-1,
// xq1 = nt q+1, xj1 = nt j-1 (only those that exist are read)
__device__ int twoloop_e(const SdParams &P, int t, int ti, int l1, int l2, int xi1, int xp1,
                         int xq1, int xj1) {
  const int s = c_rev[ti];
  if (l1 == 0 && l2 == 0) return P.stack[t][s];
  if (l1 == 0 || l2 == 0) {
    const int l = l1 + l2;
    if (l == 1) return P.bulge[1] + P.stack[t][s];
    return P.bulge[l] + P.au[t] + P.au[s];
  }
  if (l1 == 1 && l2 == 1) return P.int11[t][s][xi1 * 4 + xj1];
  if (l1 == 1 && l2 == 2) return P.int21[t][s][xi1 * 16 + xq1 * 4 + xj1];
  if (l1 == 2 && l2 == 1) return P.int21[s][t][xq1 * 16 + xi1 * 4 + xp1];
  if (l1 == 2 && l2 == 2) return P.int22[t][s][xi1 * 64 + xp1 * 16 + xq1 * 4 + xj1];
  const int d = l1 > l2 ? l1 - l2 : l2 - l1;
  const int asym = min(P.maxninio, P.ninio * d);
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

// hairpin energy of the complete hairpin: pair t, loop labels packed 2 bits
// each with the first loop label most significant
__device__ int hairpin_seq_e(const SdParams &P, const int32_t *hp_len, int t, uint32_t labs,
                             int L) {
  const int s = L == 3 ? 0 : L == 4 ? 1 : L == 6 ? 2 : -1;
  const int first = (labs >> (2 * (L - 1))) & 3, last = labs & 3;
  if (s >= 0) {
    int code = c_pair5[t];
    for (int k = 0; k < L; k++) code |= (int)((labs >> (2 * (L - 1 - k))) & 3) << (2 * (k + 1));
    code |= c_pair3[t] << (2 * (L + 1));
    for (int k = 0; k < P.nspecial[s]; k++)
      if (P.special_code[s][k] == code) return P.special_e[s][k];
  }
  return hairpin_generic_e(P, hp_len, t, L, first, last);
}

// Algorithmic work accounting (counting variant only): every min-plus term
// whose operands are finite adds 2 * (int64 additions + 1 min) INT32 slots.
#define TERM(k)                        \
  do {                                 \
    if (COUNT) ops += 2 * ((k) + 1);   \
  } while (0)

// The hot scalar tables, staged in shared memory by every fill block.
struct SmallTables {
  int32_t stack[6][6];
  int32_t mmH[6][16], mmI[6][16], mm1n[6][16], mm23[6][16];
  int32_t bulge[32], interior[32];
  int32_t au[6];
  int32_t ninio, maxninio, mlclosing, mlintern, mlbase;
};

template <int G>
__device__ __forceinline__ void seg_lexmin(int64_t &v, uint32_t &k) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const int64_t v2 = __shfl_xor_sync(FULL, v, o);
    const uint32_t k2 = __shfl_xor_sync(FULL, k, o);
    upd(v, k, v2, k2);
  }
}

// Design view for the fill: hot pointers in registers, 32-bit index math
// (sizes are limited to n <= 12000 nucleotides on the host).
struct Fv {
  int n;
  const int32_t *__restrict__ lst;
  const SdEdge *__restrict__ oe;
  const SdEdge *__restrict__ ie;
  const uint8_t *__restrict__ on;
  const uint8_t *__restrict__ in_;
  const int64_t *H;
  const uint8_t *Hk;
  const int64_t *V;
  __device__ __forceinline__ int ls(int l) const { return __ldg(lst + l); }
  __device__ __forceinline__ int w(int l) const { return __ldg(lst + l + 1) - __ldg(lst + l); }
  __device__ __forceinline__ int doff(int s) const { return (s - 1) * (n + 1) - (((s - 1) * s) >> 1); }
  // packed slot of (layer lx, slot sx) -> (layer ly, slot sy), ly > lx
  __device__ __forceinline__ int cs(int lx, int sx, int ly, int sy) const {
    return (doff(ly - lx) + lx) * SD_SLOTS + sx * SD_W + sy;
  }
  __device__ __forceinline__ int rs(int lx, int sx, int ly, int sy) const {
    return (((ly - lx) & (SD_RING - 1)) * (n + 1) + lx) * SD_SLOTS + sx * SD_W + sy;
  }
  // min path cost, 0 on the same state, +inf on another state of the same layer
  __device__ __forceinline__ int64_t Hh(int lx, int sx, int ly, int sy) const {
    if (ly == lx) return sx == sy ? 0 : SD_INF;
    return H[cs(lx, sx, ly, sy)];
  }
  __device__ __forceinline__ int nout(int v) const { return on[v]; }
  __device__ __forceinline__ int nin(int v) const { return in_[v]; }
  __device__ __forceinline__ SdEdge out(int v, int k) const { return oe[v * SD_MAXOUT + k]; }
  __device__ __forceinline__ SdEdge in(int v, int k) const { return ie[v * SD_MAXIN + k]; }
  __device__ __forceinline__ void v6(int idx, int64_t (&vv)[6]) const {
    const longlong2 *p = reinterpret_cast<const longlong2 *>(V + (int64_t)idx * 6);
    const longlong2 a = p[0], b = p[1], c = p[2];
    vv[0] = a.x;
    vv[1] = a.y;
    vv[2] = b.x;
    vv[3] = b.y;
    vv[4] = c.x;
    vv[5] = c.y;
  }
};

// lexicographic minimum over the inner pair types of vv[ti] + tab[rev ti][idx]
__device__ __forceinline__ void best_inner(const int64_t (&vv)[6], const int32_t (*tab)[16], int idx,
                                           int64_t &bv, int &bt) {
  bv = SD_INF;
  bt = 7;
#pragma unroll
  for (int ti = 0; ti < 6; ti++)
    if (fin(vv[ti])) {
      const int64_t v = vv[ti] + fx(tab[c_rev[ti]][idx]);
      if (v < bv) {
        bv = v;
        bt = ti;
      }
    }
}

// one outer type t per call: the running (value, key) minimum of Q_t
#define FOR_T(body) \
  do {              \
    body;           \
  } while (0)

// ---------------------------------------------------------------------------
// closed-interior value Q_t(x, y) for one outer type t: the loop
// closed by an outer pair of type t whose interior path runs from x (after
// the 5' nucleotide of the pair) to y (before its 3' nucleotide).  x is slot
// sx of layer lx, y slot sy of layer ly.  The work items of one layer pair are
// spread over its G threads:
//   it 0        hairpin
//   it 1..31    l1 = 0, l2 = it-1        (stack, right bulges)
//   it 32..61   l2 = 0, l1 = it-31       (left bulges)
//   it 62..90   l1 = 1, l2 = it-61       (1x1, 1x2, 1xn)
//   it 91..118  l2 = 1, l1 = it-89       (2x1, nx1)
//   it 119..121 2x2, 2x3, 3x2
//   it 122      generic internal loops through IL
//   it 123      multiloop
// Where the loop energy splits into a part that depends on the inner pair and
// a part that depends on the outer one, the best inner type comes from the
// inner cell's precomputed table.
// ---------------------------------------------------------------------------
// Item classes {first item, count, lane rotation}: the two heavy classes
// (1xn and nx1) go first on lanes 0.., bulges fill in, the small classes take
// the lanes the heavy ones leave free, so lanes of a group carry similar work.
constexpr int Q_CLASSES = 8;
__constant__ int c_qclass[Q_CLASSES][3] = {{62, 29, 0}, {91, 28, 0}, {1, 31, 1},   {32, 30, 2},
                                           {119, 3, 29}, {0, 1, 31}, {122, 1, 30}, {123, 1, 29}};

template <bool COUNT>
__device__ __forceinline__ void q_item(const Fv &F, const SdDesign &D, const SdParams &P,
                                       const SmallTables &T, int it, int x, int y, int lx, int sx,
                                       int ly, int sy, int t, int64_t &qv, uint32_t &qk,
                                       unsigned long long &ops) {
  const int g = ly - lx;
  if (it == 0) {
    if (g < 3) return;
    if (g == 3 || g == 4 || g == 6) {
      // every interior path, lexicographic label order
      int st[8], kk[8];
      int64_t cst[8];
      uint32_t labs[8];
      int depth = 0;
      st[0] = x;
      kk[0] = 0;
      cst[0] = 0;
      labs[0] = 0;
      while (depth >= 0) {
        if (depth == g) {
          const uint32_t lb = labs[g];
          FOR_T({
            upd(qv, qk, fx(hairpin_seq_e(P, D.hp_len, t, lb, g)) + cst[g], lb);
            TERM(g);
          });
          depth--;
          continue;
        }
        const int v = st[depth];
        const int k = kk[depth]++;
        if (k >= F.nout(v)) {
          depth--;
          continue;
        }
        const SdEdge e = F.out(v, k);
        const int le = lx + depth + 1;
        if (depth + 1 == g ? e.other != y : !fin(F.Hh(le, e.other - F.ls(le), ly, sy))) continue;
        st[depth + 1] = e.other;
        cst[depth + 1] = cst[depth] + e.cost;
        labs[depth + 1] = (labs[depth] << 2) | (uint32_t)e.label;
        kk[depth + 1] = 0;
        depth++;
      }
    } else {
      const int l1s = F.ls(lx + 1), l2s = F.ls(ly - 1);
      const int64_t he = fx(__ldg(&D.hp_len[g]));
      for (int a = 0; a < F.nout(x); a++) {
        const SdEdge e1 = F.out(x, a);
        for (int b = 0; b < F.nin(y); b++) {
          const SdEdge e2 = F.in(y, b);
          const int64_t h = F.Hh(lx + 1, e1.other - l1s, ly - 1, e2.other - l2s);
          if (!fin(h)) continue;
          const int64_t base = e1.cost + e2.cost + h + he;
          const uint32_t key = (uint32_t)(e1.label * 4 + e2.label);
          FOR_T({
            upd(qv, qk, base + fx(T.mmH[t][e1.label * 4 + e2.label]), key);
            TERM(3);
          });
        }
      }
    }
    return;
  }
  if (it <= 61) {  // stack and bulges: one side empty
    const bool right = it <= 31;
    const int l = right ? it - 1 : it - 31;
    if (g - l < 5) return;
    const int lo = right ? ly - l : lx + l;  // layer of the inner state that moves
    const int wo = F.w(lo);
    for (int so = 0; so < wo; so++) {
      int64_t h = 0;
      int hk = 0;
      if (l > 0) {
        const int q = right ? F.cs(lo, so, ly, sy) : F.cs(lx, sx, lo, so);
        h = F.H[q];
        if (!fin(h)) continue;
        hk = F.Hk[q];
      } else if (so != sy) {
        continue;
      }
      const int cs = right ? sx : so, ds = right ? so : sy;
      const uint32_t kb = right ? tl_key(0, l, cs, ds, 0, 0, 0, hk >> 2, hk & 3)
                                : tl_key(l, 0, cs, ds, 0, hk >> 2, hk & 3, 0, 0);
      if (l >= 2) {
        // bulge: bulge[l] + AU(t) + AU(inner); best inner type from the inner table
        const int rc = right ? F.rs(lx, sx, lo, so) : F.rs(lo, so, ly, sy);
        const int64_t pk = D.W[(int64_t)rc * SD_WN + 48];
        if (!fin(pk)) continue;
        const int64_t b2 = (pk >> 3) + h + fx(T.bulge[l]);
        const uint32_t key = kb | ((uint32_t)(pk & 7) << 8);
        FOR_T({
          upd(qv, qk, b2 + fx(T.au[t]), key);
          TERM(2);
        });
      } else {
        int64_t vv[6];
        F.v6(right ? F.cs(lx, sx, lo, so) : F.cs(lo, so, ly, sy), vv);
        const int64_t e1 = h + fx(l == 1 ? T.bulge[1] : 0);
#pragma unroll
        for (int ti = 0; ti < 6; ti++) {
          if (!fin(vv[ti])) continue;
          const int s = c_rev[ti];
          const uint32_t key = kb | ((uint32_t)ti << 8);
          FOR_T({
            upd(qv, qk, vv[ti] + e1 + fx(T.stack[t][s]), key);
            TERM(2);
          });
        }
      }
    }
    return;
  }
  if (it <= 90) {  // l1 = 1: 1x1, 1x2, 1xn
    const int l2 = it - 61;
    if (g - 1 - l2 < 5) return;
    const int ld = ly - l2, wd = F.w(ld), lds = F.ls(ld);
    const int lc = lx + 1, lcs = F.ls(lc);
    const int ld1s = F.ls(ld + 1), ly1s = F.ls(ly - 1);
    const int64_t e0 = fx(T.interior[1 + l2] + min(T.maxninio, T.ninio * (l2 - 1)));
    for (int a = 0; a < F.nout(x); a++) {
      const SdEdge ec = F.out(x, a);
      const int p = ec.label, cs = ec.other - lcs;
      for (int ds = 0; ds < wd; ds++) {
        const int d = lds + ds;
        int64_t vv[6];
        if (l2 <= 2) {
          F.v6(F.cs(lc, cs, ld, ds), vv);
          if (!(fin(vv[0]) || fin(vv[1]) || fin(vv[2]) || fin(vv[3]) || fin(vv[4]) || fin(vv[5])))
            continue;
        }
        for (int b = 0; b < F.nout(d); b++) {
          const SdEdge r1 = F.out(d, b);
          const int fR = r1.label;
          if (l2 >= 3) {
            const int64_t pk = D.W[(int64_t)F.rs(lc, cs, ld, ds) * SD_WN + p * 4 + fR];
            if (!fin(pk)) continue;
            const int64_t wv = pk >> 3;
            const int wt = (int)(pk & 7);
            const int64_t base = wv + ec.cost + r1.cost + e0;
            for (int b2 = 0; b2 < F.nin(y); b2++) {
              const SdEdge r2 = F.in(y, b2);
              const int64_t h = F.Hh(ld + 1, r1.other - ld1s, ly - 1, r2.other - ly1s);
              if (!fin(h)) continue;
              const int lR = r2.label;
              const uint32_t key = tl_key(1, l2, cs, ds, wt, p, p, fR, lR);
              const int64_t b3 = base + h + r2.cost;
              FOR_T({
                upd(qv, qk, b3 + fx(T.mm1n[t][p * 4 + lR]), key);
                TERM(5);
              });
            }
          } else if (l2 == 1) {
            if (r1.other != y) continue;
            const int64_t base = ec.cost + r1.cost;
#pragma unroll
            for (int ti = 0; ti < 6; ti++) {
              if (!fin(vv[ti])) continue;
              const int s = c_rev[ti];
              const uint32_t key = tl_key(1, 1, cs, ds, ti, p, p, fR, fR);
              FOR_T({
                upd(qv, qk, vv[ti] + base + fx(P.int11[t][s][p * 4 + fR]), key);
                TERM(3);
              });
            }
          } else {  // l2 == 2: explicit 2-edge right side
            const int m = r1.other;
            for (int b2 = 0; b2 < F.nout(m); b2++) {
              const SdEdge r2 = F.out(m, b2);
              if (r2.other != y) continue;
              const int lR = r2.label;
              const int64_t base = ec.cost + r1.cost + r2.cost;
#pragma unroll
              for (int ti = 0; ti < 6; ti++) {
                if (!fin(vv[ti])) continue;
                const int s = c_rev[ti];
                const uint32_t key = tl_key(1, 2, cs, ds, ti, p, p, fR, lR);
                FOR_T({
                  upd(qv, qk, vv[ti] + base + fx(P.int21[t][s][p * 16 + fR * 4 + lR]), key);
                  TERM(4);
                });
              }
            }
          }
        }
      }
    }
    (void)lds;
    return;
  }
  if (it <= 118) {  // l2 = 1, l1 >= 2: 2x1, nx1
    const int l1 = it - 89;
    if (g - 1 - l1 < 5) return;
    const int lc = lx + l1, wc = F.w(lc), lcs = F.ls(lc);
    const int ld = ly - 1, lds = F.ls(ld);
    const int lx1s = F.ls(lx + 1), lc1s = F.ls(lc - 1);
    const int64_t e0 = fx(T.interior[l1 + 1] + min(T.maxninio, T.ninio * (l1 - 1)));
    for (int b = 0; b < F.nin(y); b++) {
      const SdEdge er = F.in(y, b);
      const int r = er.label, ds = er.other - lds;
      for (int cs = 0; cs < wc; cs++) {
        const int c = lcs + cs;
        int64_t vv[6];
        if (l1 == 2) {
          F.v6(F.cs(lc, cs, ld, ds), vv);
          if (!(fin(vv[0]) || fin(vv[1]) || fin(vv[2]) || fin(vv[3]) || fin(vv[4]) || fin(vv[5])))
            continue;
        }
        for (int a2 = 0; a2 < F.nin(c); a2++) {
          const SdEdge p2 = F.in(c, a2);
          const int lL = p2.label;
          if (l1 >= 3) {
            const int64_t pk = D.W[(int64_t)F.rs(lc, cs, ld, ds) * SD_WN + lL * 4 + r];
            if (!fin(pk)) continue;
            const int64_t wv = pk >> 3;
            const int wt = (int)(pk & 7);
            const int64_t base = wv + er.cost + p2.cost + e0;
            for (int a = 0; a < F.nout(x); a++) {
              const SdEdge p1 = F.out(x, a);
              const int64_t h = F.Hh(lx + 1, p1.other - lx1s, lc - 1, p2.other - lc1s);
              if (!fin(h)) continue;
              const int fL = p1.label;
              const uint32_t key = tl_key(l1, 1, cs, ds, wt, fL, lL, r, r);
              const int64_t b3 = base + h + p1.cost;
              FOR_T({
                upd(qv, qk, b3 + fx(T.mm1n[t][fL * 4 + r]), key);
                TERM(5);
              });
            }
          } else {  // l1 == 2: explicit 2-edge left side
            for (int a = 0; a < F.nout(x); a++) {
              const SdEdge p1 = F.out(x, a);
              if (p1.other != p2.other) continue;
              const int fL = p1.label;
              const int64_t base = er.cost + p1.cost + p2.cost;
#pragma unroll
              for (int ti = 0; ti < 6; ti++) {
                if (!fin(vv[ti])) continue;
                const int s = c_rev[ti];
                const uint32_t key = tl_key(2, 1, cs, ds, ti, fL, lL, r, r);
                FOR_T({
                  upd(qv, qk, vv[ti] + base + fx(P.int21[s][t][r * 16 + fL * 4 + lL]), key);
                  TERM(4);
                });
              }
            }
          }
        }
      }
    }
    return;
  }
  if (it <= 121) {  // 2x2, 2x3, 3x2
    const int cls = it - 119;
    const int l1 = cls == 2 ? 3 : 2, l2 = cls == 1 ? 3 : 2;
    if (g - l1 - l2 < 5) return;
    const int lc = lx + l1, ld = ly - l2;
    const int wc = F.w(lc), wd = F.w(ld), lcs = F.ls(lc), lds = F.ls(ld);
    const int lx1s = F.ls(lx + 1), lc1s = F.ls(lc - 1), ld1s = F.ls(ld + 1), ly1s = F.ls(ly - 1);
    for (int cs = 0; cs < wc; cs++)
      for (int ds = 0; ds < wd; ds++) {
        const int c = lcs + cs, d = lds + ds;
        int64_t vv[6];
        if (cls == 0) {
          F.v6(F.cs(lc, cs, ld, ds), vv);
          if (!(fin(vv[0]) || fin(vv[1]) || fin(vv[2]) || fin(vv[3]) || fin(vv[4]) || fin(vv[5])))
            continue;
        }
        for (int a2 = 0; a2 < F.nin(c); a2++) {
          const SdEdge p2 = F.in(c, a2);
          for (int b = 0; b < F.nout(d); b++) {
            const SdEdge r1 = F.out(d, b);
            // inner part: best inner type for this (lL, fR) (2x3 / 3x2 only)
            int64_t wv = SD_INF;
            int wt = 7;
            if (cls) {
              const int64_t pk =
                  D.W[(int64_t)F.rs(lc, cs, ld, ds) * SD_WN + 16 + p2.label * 4 + r1.label];
              if (fin(pk)) {
                wv = pk >> 3;
                wt = (int)(pk & 7);
              }
            }
            if (cls && !fin(wv)) continue;
            for (int a = 0; a < F.nout(x); a++) {
              const SdEdge p1 = F.out(x, a);
              const int64_t hl = F.Hh(lx + 1, p1.other - lx1s, lc - 1, p2.other - lc1s);
              if (!fin(hl)) continue;
              for (int b2 = 0; b2 < F.nin(y); b2++) {
                const SdEdge r2 = F.in(y, b2);
                const int64_t hr = F.Hh(ld + 1, r1.other - ld1s, ly - 1, r2.other - ly1s);
                if (!fin(hr)) continue;
                const int64_t hc = p1.cost + p2.cost + r1.cost + r2.cost + hl + hr;
                if (cls) {
                  const uint32_t key =
                      tl_key(l1, l2, cs, ds, wt, p1.label, p2.label, r1.label, r2.label);
                  const int64_t b3 = wv + hc + fx(T.interior[5] + T.ninio);
                  FOR_T({
                    upd(qv, qk, b3 + fx(T.mm23[t][p1.label * 4 + r2.label]), key);
                    TERM(8);
                  });
                } else {
#pragma unroll
                  for (int ti = 0; ti < 6; ti++) {
                    if (!fin(vv[ti])) continue;
                    const int s = c_rev[ti];
                    const uint32_t key =
                        tl_key(2, 2, cs, ds, ti, p1.label, p2.label, r1.label, r2.label);
                    FOR_T({
                      upd(qv, qk,
                          vv[ti] + hc +
                              fx(P.int22[t][s][p1.label * 64 + p2.label * 16 + r1.label * 4 +
                                               r2.label]),
                          key);
                      TERM(8);
                    });
                  }
                }
              }
            }
          }
        }
      }
    return;
  }
  if (it == 122) {  // generic internal loops: mismatch edges + IL two spans below
    if (g < 11) return;
    const int l1s = F.ls(lx + 1), l2s = F.ls(ly - 1);
    for (int a = 0; a < F.nout(x); a++) {
      const SdEdge e1 = F.out(x, a);
      for (int b = 0; b < F.nin(y); b++) {
        const SdEdge e2 = F.in(y, b);
        const int r = F.rs(lx + 1, e1.other - l1s, ly - 1, e2.other - l2s);
        const int64_t il = D.IL[r];
        if (!fin(il)) continue;
        const uint32_t key = (1u << 25) | D.ILk[r] | ((uint32_t)e1.label << 6) | (uint32_t)e2.label;
        const int64_t base = il + e1.cost + e2.cost;
        FOR_T({
          upd(qv, qk, base + fx(T.mmI[t][e1.label * 4 + e2.label]), key);
          TERM(3);
        });
      }
    }
    return;
  }
  // multiloop closed by the pair
  if (g < 10) return;
  const int64_t s2 = D.S2[F.cs(lx, sx, ly, sy)];
  if (!fin(s2)) return;
  FOR_T({
    upd(qv, qk, s2 + fx(T.mlclosing + T.mlintern + T.au[t]), KEY_ML);
    TERM(1);
  });
}

// (l1', l2') pairs of the generic internal loops, l1'+l2' in [2, 26]
constexpr int IL_PAIRS = 375;

// ---------------------------------------------------------------------------
// the span kernel: G threads per layer pair (i, i+g).  With G = 1 a warp
// takes 32 layer pairs of one residue class mod 3 (so its lanes see the same
// layer types and take the same branches); otherwise consecutive groups take
// consecutive layer pairs.
// ---------------------------------------------------------------------------
template <int G>
struct FillShape {
  static constexpr int threads = G == 1 ? 96 : 128;
  static constexpr int pairs = threads / G;
  __device__ static int pair_index(int bx) {
    if (G == 1) {
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      return bx * 96 + warp + 3 * lane;
    }
    return bx * pairs + (int)threadIdx.x / G;
  }
};

template <int G, bool COUNT>
__global__ void __launch_bounds__(FillShape<G>::threads, 512 / FillShape<G>::threads)
    k_fill_span(const SdDesign *__restrict__ designs, const SdParams *__restrict__ Pp, int g,
                int nact, int items, const int32_t *__restrict__ cpre,
                unsigned long long *ops_out) {
  constexpr int NT = FillShape<G>::threads;
  __shared__ SmallTables T;
  __shared__ uint16_t s_il[IL_PAIRS];
  {
    const int32_t *src[] = {&Pp->stack[0][0], &Pp->mmH[0][0], &Pp->bulge[0], &Pp->au[0],
                            &Pp->ninio};
    int32_t *dst[] = {&T.stack[0][0], &T.mmH[0][0], &T.bulge[0], &T.au[0], &T.ninio};
    const int cnt[] = {36, 4 * 96, 64, 6, 5};
#pragma unroll
    for (int q = 0; q < 5; q++)
      for (int k = threadIdx.x; k < cnt[q]; k += NT) dst[q][k] = src[q][k];
    for (int k = threadIdx.x; k < 27 * 27; k += NT) {
      const int l1p = k / 27, l2p = k % 27;
      if (l1p + l2p < 2 || l1p + l2p > SD_MAXTWO - 4) continue;
      // rank of (l1p, l2p) among the admissible pairs in row-major order
      int r = 0;
      for (int a = 0; a < l1p; a++) r += (SD_MAXTWO - 4 - a + 1) - (a < 2 ? 2 - a : 0);
      r += l2p - (l1p < 2 ? 2 - l1p : 0);
      s_il[r] = (uint16_t)(l1p | (l2p << 5));
    }
  }
  __syncthreads();
  unsigned long long ops = 0;
  const int lane = threadIdx.x & 31, sub = lane & (G - 1);
  // work queue of the span: the layer pairs of the nact designs still running
  // (designs sorted by length, longest first), design d owning items
  // [cpre[d] - d*g, cpre[d+1] - (d+1)*g)
  const int q = FillShape<G>::pair_index(blockIdx.x);
  int dsel = 0;
  if (q < items) {
    int lo = 0, hi = nact - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(&cpre[mid]) - mid * g <= q) lo = mid;
      else hi = mid - 1;
    }
    dsel = lo;
  }
  const SdDesign &D = designs[dsel];
  const SdParams &P = *Pp;
  const int n = D.n;
  const int i = q - (__ldg(&cpre[dsel]) - dsel * g);
  const bool active = q < items && g <= n && i >= 0 && i <= n - g;
  if (__all_sync(FULL, !active)) return;
  const int j = i + g;
  Fv F;
  F.n = n;
  F.lst = D.lstart;
  F.oe = D.out;
  F.ie = D.in;
  F.on = D.out_cnt;
  F.in_ = D.in_cnt;
  F.H = D.H;
  F.Hk = D.Hk;
  F.V = D.V;
  int a0 = 0, wa = 0, b0 = 0, wb = 0;
  if (active) {
    a0 = F.ls(i);
    wa = F.ls(i + 1) - a0;
    b0 = F.ls(j);
    wb = F.ls(j + 1) - b0;
  }
  const int cell = active ? (F.doff(g) + i) * SD_SLOTS : 0;
  const int rcell = ((g & (SD_RING - 1)) * (n + 1) + i) * SD_SLOTS;
  const int64_t mlb = fx(T.mlbase);
  const int js = active ? F.ls(j - 1) : 0;  // first state on layer j-1
  const int i1s = active ? F.ls(i + 1) : 0;

  int64_t Bs[SD_SLOTS], PSs[SD_SLOTS];
#pragma unroll
  for (int s = 0; s < SD_SLOTS; s++) {
    Bs[s] = SD_INF;
    PSs[s] = SD_INF;
  }
#pragma unroll 1
  for (int s = 0; s < SD_SLOTS; s++) {
    const int sa = s / SD_W, sb = s % SD_W;
    const bool ok = active && sa < wa && sb < wb;
    const int a = a0 + sa, b = b0 + sb;
    // gap cell (every thread of the group; at most a few in-edges)
    if (ok) {
      int64_t hv = SD_INF;
      uint32_t hk = KEY_NONE;
      for (int k = 0; k < F.nin(b); k++) {
        const SdEdge e = F.in(b, k);
        int64_t hp;
        int f;
        if (g == 1) {
          hp = e.other == a ? 0 : SD_INF;
          f = e.label;
        } else {
          const int q = F.cs(i, sa, j - 1, e.other - js);
          hp = F.H[q];
          f = F.Hk[q] >> 2;
        }
        if (!fin(hp)) continue;
        upd(hv, hk, hp + e.cost, (uint32_t)(f * 4 + e.label));
        TERM(1);
      }
      settle(hv, hk);
      if (sub == 0) {
        D.H[cell + s] = hv;
        D.Hk[cell + s] = (uint8_t)(hk & 15);
      }
    }
    // Ihat: inner pair (c,d) one nucleotide inside (a,b) and its loop-side
    // mismatch; key fields: slot of c, slot of d, inner type, lL, fR
    {
      int64_t iv = SD_INF;
      uint32_t ik = KEY_NONE;
      if (ok && g >= 7) {
        const int no = F.nout(a), ni = F.nin(b);
        for (int q = sub; q < no * ni; q += G) {
          const int k2 = q % ni, k1 = q / ni;
          const SdEdge e1 = F.out(a, k1), e2 = F.in(b, k2);
          const int cs = e1.other - i1s, ds = e2.other - js;
          const int64_t pk =
              D.W[(int64_t)F.rs(i + 1, cs, j - 1, ds) * SD_WN + 32 + e1.label * 4 + e2.label];
          if (!fin(pk)) continue;
          const uint32_t key = ((uint32_t)cs << 13) | ((uint32_t)ds << 11) |
                               ((uint32_t)(pk & 7) << 8) | ((uint32_t)e1.label << 4) |
                               ((uint32_t)e2.label << 2);
          upd(iv, ik, (pk >> 3) + e1.cost + e2.cost, key);
          TERM(3);
        }
      }
      seg_lexmin<G>(iv, ik);
      settle(iv, ik);
      if (ok && sub == 0) {
        D.Ihat[rcell + s] = iv;
        D.Ihk[rcell + s] = ik;
      }
    }
    // IL: generic internal loops l1 = l1'+2, l2 = l2'+2 around (a,b)
    {
      int64_t lv = SD_INF;
      uint32_t lk = KEY_NONE;
      if (ok && g >= 9) {
        for (int q = sub; q < IL_PAIRS; q += G) {
          const int pr = s_il[q];
          const int l1p = pr & 31, l2p = pr >> 5;
          const int lc = i + l1p, ld = j - l2p;
          if (ld - lc < 7) continue;
          const int dd = l1p > l2p ? l1p - l2p : l2p - l1p;
          const int64_t e = fx(T.interior[l1p + l2p + 4] + min(T.maxninio, T.ninio * dd));
          const uint32_t kl = ((uint32_t)(l1p + l2p + 4) << 20) | ((uint32_t)(l1p + 2) << 15);
          const int wc = F.w(lc), wd = F.w(ld);
          for (int cs = 0; cs < wc; cs++) {
            const int64_t hl = F.Hh(i, sa, lc, cs);
            if (!fin(hl)) continue;
            for (int ds = 0; ds < wd; ds++) {
              const int64_t hr = F.Hh(ld, ds, j, sb);
              if (!fin(hr)) continue;
              const int r = F.rs(lc, cs, ld, ds);
              const int64_t v = D.Ihat[r];
              if (!fin(v)) continue;
              upd(lv, lk, hl + v + hr + e, kl | D.Ihk[r]);
              TERM(3);
            }
          }
        }
      }
      seg_lexmin<G>(lv, lk);
      settle(lv, lk);
      if (ok && sub == 0) {
        D.IL[rcell + s] = lv;
        D.ILk[rcell + s] = lk;
      }
    }
    // typed closed values (every thread of the group) and Eq. (branch)
    int64_t vv[6];
    {
      int64_t B = SD_INF;
      uint32_t Bk = KEY_NONE;
#pragma unroll
      for (int t = 0; t < 6; t++) {
        int64_t v = SD_INF;
        uint32_t vk = KEY_NONE;
        if (ok && g >= 5) {
          for (int k1 = 0; k1 < F.nout(a); k1++) {
            const SdEdge e1 = F.out(a, k1);
            if (e1.label != c_pair5[t]) continue;
            for (int k2 = 0; k2 < F.nin(b); k2++) {
              const SdEdge e2 = F.in(b, k2);
              if (e2.label != c_pair3[t]) continue;
              const int r = F.rs(i + 1, e1.other - i1s, j - 1, e2.other - js) * 6 + t;
              const int64_t q = D.Q[r];
              if (!fin(q)) continue;
              upd(v, vk, q + e1.cost + e2.cost, ((uint32_t)k2 << 27) | D.Qk[r]);
              TERM(2);
            }
          }
        }
        settle(v, vk);
        vv[t] = v;
        if (ok && sub == t % G) {
          D.V[(int64_t)(cell + s) * 6 + t] = v;
          D.Vk[(int64_t)(cell + s) * 6 + t] = vk;
        }
        if (fin(v)) {
          upd(B, Bk, v + fx(T.mlintern + T.au[t]), (uint32_t)t);
          TERM(1);
        }
      }
      settle(B, Bk);
      if (ok && sub == 0) {
        D.Bv[cell + s] = B;
        D.Bk[cell + s] = (uint8_t)(Bk & 7);
      }
      Bs[s] = B;
    }
    // inner tables of this cell for the two-loops that will enclose it
    if (ok) {
      const int im = D.in_mask[a], om = D.out_mask[b];
      int64_t *Wc = D.W + (int64_t)(rcell + s) * SD_WN;
      for (int q = sub; q < SD_WN; q += G) {
        int64_t bv = SD_INF;
        int bt = 7;
        if (g >= 5) {
          if (q < 48) {
            const int tab = q >> 4, li = (q >> 2) & 3, lo = q & 3;
            if (((im >> li) & 1) && ((om >> lo) & 1))
              best_inner(vv, tab == 0 ? T.mm1n : tab == 1 ? T.mm23 : T.mmI, lo * 4 + li, bv, bt);
          } else {
#pragma unroll
            for (int ti = 0; ti < 6; ti++)
              if (fin(vv[ti])) {
                const int64_t v = vv[ti] + fx(T.au[c_rev[ti]]);
                if (v < bv) {
                  bv = v;
                  bt = ti;
                }
              }
          }
        }
        Wc[q] = fin(bv) ? bv * 8 + bt : SD_INF;
      }
    }
  }
  // Eq. (sparse2) for every slot: edge extensions, then splits at retained
  // candidates (the group splits the candidate list)
#pragma unroll 1
  for (int s = 0; s < SD_SLOTS; s++) {
    const int sa = s / SD_W, sb = s % SD_W;
    const bool ok = active && sa < wa && sb < wb;
    const int a = a0 + sa, b = b0 + sb;
    int64_t s2 = SD_INF;
    uint32_t s2k = KEY_NONE;
    if (ok) {
      if (g >= 2 && sub == 0)
        for (int k = 0; k < F.nin(b); k++) {
          const SdEdge e = F.in(b, k);
          const int64_t v = D.S2[F.cs(i, sa, j - 1, e.other - js)];
          if (!fin(v)) continue;
          upd(s2, s2k, v + e.cost + mlb, (uint32_t)k);
          TERM(2);
        }
      const int cnt = D.cand_cap ? min(D.cand_cnt[b], __ldg(&D.cand_cap[b])) : D.cand_cnt[b];
      const int64_t off = D.cand_off[b];
      for (int k = sub; k < cnt; k += G) {
        const int c = D.cand_c[off + k];
        const int lc = __ldg(&D.layer[c]);
        if (lc <= i) break;  // entries are in decreasing layer order
        const int64_t v = D.S1[F.cs(i, sa, lc, c - F.ls(lc))];
        if (!fin(v)) continue;
        upd(s2, s2k, v + D.cand_B[off + k], KEY_SPLIT | (uint32_t)c);
        TERM(1);
      }
    }
    seg_lexmin<G>(s2, s2k);
    settle(s2, s2k);
    if (ok && sub == 0) {
      D.S2[cell + s] = s2;
      D.S2k[cell + s] = s2k;
      // P_S (Eq. partitionable with S) and S1 = min(B, P_S); key classes:
      // 0 direct branch, 1 left peel, 2 right peel, 3 two-branch value
      int64_t ps = s2;
      uint32_t psk = fin(s2) ? (3u << 4) : KEY_NONE;
      if (g >= 2) {
        for (int k = 0; k < F.nout(a); k++) {
          const SdEdge e = F.out(a, k);
          const int64_t v = D.S1[F.cs(i + 1, e.other - i1s, j, sb)];
          if (!fin(v)) continue;
          upd(ps, psk, v + e.cost + mlb, (1u << 4) | (uint32_t)k);
          TERM(2);
        }
        for (int k = 0; k < F.nin(b); k++) {
          const SdEdge e = F.in(b, k);
          const int64_t v = D.S1[F.cs(i, sa, j - 1, e.other - js)];
          if (!fin(v)) continue;
          upd(ps, psk, v + e.cost + mlb, (2u << 4) | (uint32_t)k);
          TERM(2);
        }
      }
      settle(ps, psk);
      int64_t s1 = ps;
      uint32_t s1k = psk;
      if (fin(Bs[s])) upd(s1, s1k, Bs[s], 0u);
      D.S1[cell + s] = s1;
      D.S1k[cell + s] = s1k;
      PSs[s] = ps;
    }
  }
  // candidate appends (Eq. candidates); the list of b is in decreasing layer
  // order and states of one layer are appended in descending id order
  if (active && sub == 0)
    for (int sb = 0; sb < wb; sb++) {
      const int b = b0 + sb;
      int cnt = D.cand_cnt[b];
      const int64_t off = D.cand_off[b];
      const int cap = D.cand_cap ? __ldg(&D.cand_cap[b]) : 0x7fffffff;
      for (int sa = wa - 1; sa >= 0; sa--) {
        const int s = sa * SD_W + sb;
        if (Bs[s] < PSs[s]) {
          if (cnt < cap) {
            D.cand_c[off + cnt] = a0 + sa;
            D.cand_B[off + cnt] = Bs[s];
          } else {
            D.tb[3] = 1;  // presized room exceeded: this run is repeated
          }
          cnt++;
        }
      }
      D.cand_cnt[b] = cnt;
    }
  // closed-interior values for the pairs two spans up
#pragma unroll 1
  for (int s = 0; s < SD_SLOTS; s++) {
    const int sa = s / SD_W, sb = s % SD_W;
    const bool ok = active && sa < wa && sb < wb;
    const int x = a0 + sa, y = b0 + sb;
    int tmask = 0;
    if (ok) {
      const int im = D.in_mask[x], om = D.out_mask[y];
#pragma unroll
      for (int t = 0; t < 6; t++)
        if (((im >> c_pair5[t]) & 1) && ((om >> c_pair3[t]) & 1)) tmask |= 1 << t;
    }
    // one outer type at a time (the types of a layer pair are the same for
    // all threads of its group); types that cannot close (x, y) stay +inf
#pragma unroll 1
    for (int t = 0; t < 6; t++) {
      int64_t qv = SD_INF;
      uint32_t qk = KEY_NONE;
      if ((tmask >> t) & 1)
        for (int cl = 0; cl < Q_CLASSES; cl++) {
          const int st = c_qclass[cl][0], cnt = c_qclass[cl][1], rot = c_qclass[cl][2] % G;
          for (int k = (sub - rot + G) % G; k < cnt; k += G)
            q_item<COUNT>(F, D, P, T, st + k, x, y, i, sa, j, sb, t, qv, qk, ops);
        }
      if (__any_sync(FULL, (tmask >> t) & 1)) seg_lexmin<G>(qv, qk);
      settle(qv, qk);
      if (ok && sub == 0) {
        D.Q[(int64_t)(rcell + s) * 6 + t] = qv;
        D.Qk[(int64_t)(rcell + s) * 6 + t] = qk;
      }
    }
  }
  if (COUNT && active && ops) atomicAdd(&ops_out[dsel], ops);
}

// ---------------------------------------------------------------------------
// exterior suffix values (Sec. 5 final-column exterior DP), one block per
// design; key: unpaired out-edge index, or KEY_SPLIT | b*8 + type
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_exterior(const SdDesign *__restrict__ designs,
                                                  const SdParams *__restrict__ Pp) {
  const SdDesign &D = designs[blockIdx.x];
  const SdParams &P = *Pp;
  __shared__ int64_t smv[8];
  __shared__ uint32_t smk[8];
  Lat G(D);
  const int n = D.n, N = D.N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    D.Ext[N - 1] = 0;
    D.Extk[N - 1] = KEY_NONE;
  }
  __syncthreads();
  for (int k = n - 1; k >= 0; k--) {
    for (int a = G.lstart(k); a < G.lstart(k + 1); a++) {
      int64_t bv = SD_INF;
      uint32_t bk = KEY_NONE;
      if ((int)threadIdx.x < G.nout(a)) {
        const SdEdge e = G.out(a, threadIdx.x);
        const int64_t x = D.Ext[e.other];
        if (fin(x)) upd(bv, bk, x + e.cost, threadIdx.x);
      }
      for (int b = G.lstart(k + 1) + threadIdx.x; b < N; b += blockDim.x) {
        const int lb = G.layer(b);
        if (lb - k < 5) continue;
        const int64_t eb = D.Ext[b];
        if (!fin(eb)) continue;
        const int64_t cs = G.slot(a, b, k, lb) * 6;
        for (int t = 0; t < 6; t++) {
          const int64_t v = D.V[cs + t];
          if (fin(v)) upd(bv, bk, v + fx(P.au[t]) + eb, KEY_SPLIT | ((uint32_t)b << 3) | t);
        }
      }
      warp_lexmin(bv, bk);
      if (lane == 0) {
        smv[w] = bv;
        smk[w] = bk;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); q++) upd(bv, bk, smv[q], smk[q]);
        settle(bv, bk);
        D.Ext[a] = bv;
        D.Extk[a] = bk;
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// traceback: follows the stored canonical keys (one thread per design) and
// re-checks every step's value, accumulating the loop energies and codon costs
// ---------------------------------------------------------------------------
struct Tb {
  const SdDesign &D;
  const SdParams &P;
  Lat G;
  int64_t energy, pathcost;
  int err;
  int sp;
  __device__ Tb(const SdDesign &d, const SdParams &p)
      : D(d), P(p), G(d), energy(0), pathcost(0), err(0), sp(0) {}

  __device__ void emit(int from, int label, int64_t cost) {
    const int pos = G.layer(from);
    if (pos < 0 || pos >= D.n || D.mrna[pos] != 0) {
      err = 2;
      return;
    }
    D.mrna[pos] = "ACGU"[label];
    pathcost += cost;
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
  // canonical min-cost path x -> y: out-edges in label order, greedy
  __device__ void gap(int x, int y) {
    const int ly = G.layer(y);
    while (x != y && !err) {
      const int64_t v = G.Hp(x, y);
      int moved = 0;
      for (int k = 0; k < G.nout(x); k++) {
        const SdEdge e = G.out(x, k);
        if (G.layer(e.other) > ly) continue;
        const int64_t h = G.Hp(e.other, y);
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
  // realise the unpaired side x -> y of len edges with first / last labels
  // f / l; returns its cost (+inf if it does not exist)
  __device__ int64_t side(int x, int y, int len, int f, int l) {
    if (len == 0) return x == y ? 0 : SD_INF;
    const int k1 = G.out_with_label(x, f);
    if (k1 < 0) return SD_INF;
    const SdEdge e1 = G.out(x, k1);
    if (len == 1) {
      if (e1.other != y) return SD_INF;
      emit(x, e1.label, e1.cost);
      return e1.cost;
    }
    if (len == 2) {
      const int k2 = G.out_with_label(e1.other, l);
      if (k2 < 0) return SD_INF;
      const SdEdge e2 = G.out(e1.other, k2);
      if (e2.other != y) return SD_INF;
      emit(x, e1.label, e1.cost);
      emit(e1.other, e2.label, e2.cost);
      return e1.cost + e2.cost;
    }
    int64_t best = SD_INF;
    for (int q = 0; q < G.nin(y); q++) {
      const SdEdge ei = G.in(y, q);
      if (ei.label != l) continue;
      const int64_t h = G.Hp(e1.other, ei.other);
      if (fin(h)) best = min(best, e1.cost + h + ei.cost);
    }
    for (int q = 0; q < G.nin(y); q++) {
      const SdEdge ei = G.in(y, q);
      if (ei.label != l) continue;
      const int64_t h = G.Hp(e1.other, ei.other);
      if (fin(h) && e1.cost + h + ei.cost == best) {
        emit(x, e1.label, e1.cost);
        gap(e1.other, ei.other);
        emit(ei.other, ei.label, ei.cost);
        return best;
      }
    }
    return SD_INF;
  }

  __device__ void trace_V(int a, int b, int t) {
    const int la = G.layer(a), lb = G.layer(b);
    const int64_t s = G.slot(a, b, la, lb);
    const int64_t v = D.V[s * 6 + t];
    const uint32_t key = D.Vk[s * 6 + t];
    const int kx = G.out_with_label(a, c_pair5[t]);
    const int ky = key >> 27;
    if (!fin(v) || kx < 0 || ky >= G.nin(b)) {
      err = 7;
      return;
    }
    const SdEdge ex = G.out(a, kx), ey = G.in(b, ky);
    const int a1 = ex.other, b1 = ey.other;
    const int lx = la + 1, ly = lb - 1, L = ly - lx;
    set_pair(la, lb - 1);
    emit(a, ex.label, ex.cost);
    emit(b1, ey.label, ey.cost);
    const uint32_t q = key & KEY_QMASK;
    const int cls = q >> 25;
    int64_t got = SD_INF;
    if (cls == 0) {  // hairpin
      if (L == 3 || L == 4 || L == 6) {
        int x = a1;
        int64_t c = 0;
        for (int k = 0; k < L && x >= 0; k++) {
          const int lab = (q >> (2 * (L - 1 - k))) & 3;
          const int kk = G.out_with_label(x, lab);
          if (kk < 0) {
            x = -1;
            break;
          }
          const SdEdge e = G.out(x, kk);
          emit(x, e.label, e.cost);
          c += e.cost;
          x = e.other;
        }
        if (x == b1) {
          const int e = hairpin_seq_e(P, D.hp_len, t, q & 0xfff, L);
          energy += e;
          got = fx(e) + c;
        }
      } else {
        const int f = (q >> 2) & 3, l = q & 3;
        const int64_t c = side(a1, b1, L, f, l);
        if (fin(c)) {
          const int e = hairpin_generic_e(P, D.hp_len, t, L, f, l);
          energy += e;
          got = fx(e) + c;
        }
      }
    } else if (cls == 1) {  // two-loop
      const int l = (q >> 20) & 31, l1 = (q >> 15) & 31, l2 = l - l1;
      const int cs = (q >> 13) & 3, ds = (q >> 11) & 3, ti = (q >> 8) & 7;
      const int fL = (q >> 6) & 3, lL = (q >> 4) & 3, fR = (q >> 2) & 3, lR = q & 3;
      const int lc = lx + l1, ld = ly - l2;
      if (l2 >= 0 && ld - lc >= 5 && ti < 6) {
        const int c = G.lstart(lc) + cs, d = G.lstart(ld) + ds;
        const int64_t cl = side(a1, c, l1, fL, lL);
        const int64_t cr = side(d, b1, l2, fR, lR);
        const int64_t vi = G.Vt(c, d, ti);
        if (fin(cl) && fin(cr) && fin(vi)) {
          const int e = twoloop_e(P, t, ti, l1, l2, fL, lL, fR, lR);
          energy += e;
          got = fx(e) + cl + cr + vi;
          push(1, c, d, ti);
        }
      }
    } else {  // multiloop
      const int64_t s2 = G.S2(a1, b1);
      if (fin(s2)) {
        energy += P.mlclosing + P.mlintern + P.au[t];
        got = s2 + fx(P.mlclosing + P.mlintern + P.au[t]);
        push(3, a1, b1, 0);
      }
    }
    if (!fin(got) || got + ex.cost + ey.cost != v) err = 8;
  }
  __device__ void trace_B(int a, int b) {
    const int64_t s = G.slot(a, b, G.layer(a), G.layer(b));
    const int t = D.Bk[s];
    const int64_t v = t < 6 ? G.Vt(a, b, t) : SD_INF;
    if (!fin(v) || v + fx(P.mlintern + P.au[t]) != D.Bv[s]) {
      err = 9;
      return;
    }
    energy += P.mlintern + P.au[t];
    trace_V(a, b, t);
  }
  __device__ void trace_S2(int a, int b) {
    const int la = G.layer(a);
    while (!err) {
      const int lb = G.layer(b);
      if (lb <= la) {
        err = 10;
        return;
      }
      const int64_t s = G.slot(a, b, la, lb);
      const int64_t v = D.S2[s];
      const uint32_t key = D.S2k[s];
      if (!fin(v)) {
        err = 10;
        return;
      }
      if (key < KEY_SPLIT) {
        if ((int)key >= G.nin(b)) {
          err = 10;
          return;
        }
        const SdEdge e = G.in(b, key);
        const int64_t x = G.S2(a, e.other);
        if (!fin(x) || x + e.cost + fx(P.mlbase) != v) {
          err = 10;
          return;
        }
        emit(e.other, e.label, e.cost);
        energy += P.mlbase;
        b = e.other;
        continue;
      }
      const int c = key & (KEY_SPLIT - 1);
      if (c >= D.N) {
        err = 11;
        return;
      }
      const int64_t x = G.S1(a, c);
      const int lc = G.layer(c);
      const int64_t bc = (lb - lc >= 5) ? D.Bv[G.slot(c, b, lc, lb)] : SD_INF;
      if (!fin(x) || !fin(bc) || x + bc != v) {
        err = 11;
        return;
      }
      push(2, a, c, 0);
      push(4, c, b, 0);
      return;
    }
  }
  __device__ void trace_S1(int a, int b) {
    const int64_t mlb = fx(P.mlbase);
    while (!err) {
      const int la = G.layer(a), lb = G.layer(b);
      if (lb <= la) {
        err = 12;
        return;
      }
      const int64_t s = G.slot(a, b, la, lb);
      const int64_t v = D.S1[s];
      const uint32_t key = D.S1k[s];
      if (!fin(v)) {
        err = 12;
        return;
      }
      const int cls = key >> 4, k = key & 15;
      if (cls == 0) {
        if (D.Bv[s] != v) err = 12;
        else trace_B(a, b);
        return;
      }
      if (cls == 1) {
        if (k >= G.nout(a)) {
          err = 13;
          return;
        }
        const SdEdge e = G.out(a, k);
        const int64_t x = G.S1(e.other, b);
        if (!fin(x) || x + e.cost + mlb != v) {
          err = 13;
          return;
        }
        emit(a, e.label, e.cost);
        energy += P.mlbase;
        a = e.other;
        continue;
      }
      if (cls == 2) {
        if (k >= G.nin(b)) {
          err = 13;
          return;
        }
        const SdEdge e = G.in(b, k);
        const int64_t x = G.S1(a, e.other);
        if (!fin(x) || x + e.cost + mlb != v) {
          err = 13;
          return;
        }
        emit(e.other, e.label, e.cost);
        energy += P.mlbase;
        b = e.other;
        continue;
      }
      if (D.S2[s] != v) err = 13;
      else trace_S2(a, b);
      return;
    }
  }
  __device__ void run() {
    const int N = D.N;
    int a = 0;
    const int tstate = N - 1;
    if (!fin(D.Ext[0])) {
      err = 14;
      return;
    }
    while (a != tstate && !err) {
      const int64_t v = D.Ext[a];
      const uint32_t key = D.Extk[a];
      if (key < KEY_SPLIT) {
        if ((int)key >= G.nout(a)) {
          err = 15;
          break;
        }
        const SdEdge e = G.out(a, key);
        if (D.Ext[e.other] + e.cost != v) {
          err = 15;
          break;
        }
        emit(a, e.label, e.cost);
        a = e.other;
      } else {
        const int b = (key & (KEY_SPLIT - 1)) >> 3, t = key & 7;
        const int64_t x = (b < N && t < 6) ? G.Vt(a, b, t) : SD_INF;
        if (!fin(x) || x + fx(P.au[t]) + D.Ext[b] != v) {
          err = 15;
          break;
        }
        energy += P.au[t];
        push(1, a, b, t);
        a = b;
      }
    }
    while (sp > 0 && !err) {
      const int32_t *s = D.tb_stack + 4 * --sp;
      const int type = s[0], x = s[1], y = s[2], t = s[3];
      if (type == 1) trace_V(x, y, t);
      else if (type == 2) trace_S1(x, y);
      else if (type == 3) trace_S2(x, y);
      else trace_B(x, y);
    }
    for (int k = 0; k < D.n && !err; k++)
      if (D.mrna[k] == 0) err = 16;
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
  if (blockIdx.x == 0 && threadIdx.x == 0) D.tb[3] = 0;
}

// Retained candidates of one design by (codon position of the right endpoint,
// span band): band = floor(log2(span)) - 2 clamped to [0, 7], i.e. spans
// 5-7, 8-15, ..., 256-511, >= 512.  hist: A * 8 counters, zeroed by the caller.
__global__ void k_retention(const SdDesign *__restrict__ designs, int item, int32_t *hist) {
  const SdDesign &D = designs[item];
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < D.N; b += gridDim.x * blockDim.x) {
    const int lb = D.layer[b];
    if (lb < 1) continue;
    const int k = (lb - 1) / 3;
    const int cnt = D.cand_cap ? min(D.cand_cnt[b], D.cand_cap[b]) : D.cand_cnt[b];
    const int64_t off = D.cand_off[b];
    for (int q = 0; q < cnt; q++) {
      const int span = lb - D.layer[D.cand_c[off + q]];
      const int band = min(7, max(0, 31 - __clz(span) - 2));
      atomicAdd(&hist[k * 8 + band], 1);
    }
  }
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

// One launch per span over the span's work queue.  ns: lengths of the
// designs in device order (non-increasing); cpre: their prefix sums of n+1.
template <int G, bool COUNT>
void launch_fill_g(const SdDesign *d_designs, int count, const int *ns, const int32_t *d_cpre,
                   const SdParams *d_params, cudaStream_t st, unsigned long long *d_ops) {
  constexpr int per_block = G == 1 ? 96 : FillShape<G>::pairs;
  int nact = count;
  int64_t cp = 0;
  for (int d = 0; d < count; d++) cp += ns[d] + 1;
  const int max_n = count > 0 ? ns[0] : 0;
  for (int g = 1; g <= max_n; g++) {
    while (nact > 0 && ns[nact - 1] < g) {
      nact--;
      cp -= ns[nact] + 1;
    }
    const int64_t items = cp - (int64_t)nact * g;
    if (items <= 0) break;
    dim3 grid((unsigned)((items + per_block - 1) / per_block));
    k_fill_span<G, COUNT><<<grid, FillShape<G>::threads, 0, st>>>(d_designs, d_params, g, nact,
                                                                  (int)items, d_cpre, d_ops);
  }
}

template <bool COUNT>
int launch_fill(int G, const SdDesign *d_designs, int count, const int *ns, const int32_t *d_cpre,
                const SdParams *d_params, cudaStream_t st, unsigned long long *d_ops) {
  switch (G) {
    case 1: launch_fill_g<1, COUNT>(d_designs, count, ns, d_cpre, d_params, st, d_ops); break;
    case 8: launch_fill_g<8, COUNT>(d_designs, count, ns, d_cpre, d_params, st, d_ops); break;
    case 32: launch_fill_g<32, COUNT>(d_designs, count, ns, d_cpre, d_params, st, d_ops); break;
    default: return -1;
  }
  return 0;
}

}  // namespace

extern "C" int sd_k_retention(const SdDesign *d_designs, int item, int32_t *d_hist, int ncodons,
                              void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_hist, 0, sizeof(int32_t) * 8 * (ncodons > 0 ? ncodons : 1), st) !=
      cudaSuccess)
    return -1;
  k_retention<<<64, 256, 0, st>>>(d_designs, item, d_hist);
  if (cudaGetLastError() != cudaSuccess) return -1;
  return cudaStreamSynchronize(st) == cudaSuccess ? 0 : -1;
}

extern "C" int sd_k_count(const SdDesign *d_designs, int count, int64_t *d_out, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_out, 0, sizeof(int64_t) * 4 * count, st) != cudaSuccess) return -1;
  k_count<<<dim3(64, count), 256, 0, st>>>(d_designs, (unsigned long long *)d_out);
  if (cudaGetLastError() != cudaSuccess) return -1;
  return cudaStreamSynchronize(st) == cudaSuccess ? 0 : -1;
}

// Counting pass: the same fill with algorithmic-work counters (INT32 slots
// per design, see TERM); the result tables are identical to sd_k_run's.
extern "C" int sd_k_count_ops(const SdDesign *d_designs, int count, const int *ns,
                              const int32_t *d_cpre, const SdParams *d_params,
                              unsigned long long *d_ops, void *stream, int group) {
  cudaStream_t st = (cudaStream_t)stream;
  if (count <= 0) return 0;
  if (cudaMemsetAsync(d_ops, 0, sizeof(unsigned long long) * count, st) != cudaSuccess) return -1;
  k_clear_cand<<<dim3(8, count), 256, 0, st>>>(d_designs);
  if (launch_fill<true>(group, d_designs, count, ns, d_cpre, d_params, st, d_ops)) return -1;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

extern "C" int sd_k_run(const SdDesign *d_designs, int count, const int *ns, const int32_t *d_cpre,
                        const SdParams *d_params, void *stream, int64_t *launches,
                        void *const *events, int group) {
  cudaStream_t st = (cudaStream_t)stream;
  if (count <= 0) {
    if (launches) *launches = 0;
    return 0;
  }
  k_clear_cand<<<dim3(8, count), 256, 0, st>>>(d_designs);
  if (events) cudaEventRecord((cudaEvent_t)events[0], st);
  if (launch_fill<false>(group, d_designs, count, ns, d_cpre, d_params, st, nullptr)) return -1;
  if (events) cudaEventRecord((cudaEvent_t)events[1], st);
  k_exterior<<<count, 256, 0, st>>>(d_designs, d_params);
  if (events) cudaEventRecord((cudaEvent_t)events[2], st);
  k_traceback<<<count, 128, 0, st>>>(d_designs, d_params);
  if (events) cudaEventRecord((cudaEvent_t)events[3], st);
  if (launches) *launches = (int64_t)ns[0] + 3;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
