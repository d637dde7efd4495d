// sd_kernels.cu -- sm_103a kernels of the exact codon-lattice design DP.
//
// Span wavefront (Algorithm 1, Sec. 5).  One launch per span g processes every
// layer pair (i, i+g) of every design in the batch (a work queue over
// (design, layer pair), longest design first), one group of 8, 16 or 32
// threads per layer pair.  The paper separates closed/gap values, multiloop
// values and exterior values by barriers; here all phases of one layer pair run
// in the group that owns it, because each only reads smaller spans or the same
// cell:
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
  const int32_t *__restrict__ lay;
  const SdFlatEdge *__restrict__ fo;
  const int32_t *__restrict__ fo_off;
  const SdFlatEdge *__restrict__ fi;
  const int32_t *__restrict__ fi_off;
  __device__ __forceinline__ int ls(int l) const { return __ldg(lst + l); }
  __device__ __forceinline__ int layer(int v) const { return __ldg(lay + v); }
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

// Gap values of the two ends of a layer pair, staged in shared memory per
// group: hl[l][c*2 + s] = H(slot s of layer i -> slot c of layer i+l),
// hr[l][c*2 + s] = H(slot c of layer j-l -> slot s of layer j), l < SD_GAPW,
// with the (first, last) label keys; the two-loop options read them many times.
constexpr int SD_GAPW = SD_MAXTWO + 1;
struct GapStage {
  int64_t hl[SD_GAPW][4], hr[SD_GAPW][4];
  uint8_t hlk[SD_GAPW][4], hrk[SD_GAPW][4];
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

// lexicographic minimum over the inner pair types of vv[ti] + AU(rev ti)
__device__ __forceinline__ void best_au(const int64_t (&vv)[6], const int32_t *au, int64_t &bv,
                                        int &bt) {
  bv = SD_INF;
  bt = 7;
#pragma unroll
  for (int ti = 0; ti < 6; ti++)
    if (fin(vv[ti])) {
      const int64_t v = vv[ti] + fx(au[c_rev[ti]]);
      if (v < bv) {
        bv = v;
        bt = ti;
      }
    }
}

// All outer pair types of one closed-interior cell at once: (qv[t], qk[t]) is
// the running (value, key) minimum of Q_t for every t in the type mask tm
// (the same for every thread of a group).  tab(t) is the outer-type part of
// the loop energy; the rest of the term is shared by the types.
template <bool COUNT, class Tab>
__device__ __forceinline__ void upd6(int64_t (&qv)[6], uint32_t (&qk)[6], int tm, int64_t base,
                                     uint32_t key, int nadd, unsigned long long &ops,
                                     const Tab &tab) {
#pragma unroll
  for (int t = 0; t < 6; t++)
    if ((tm >> t) & 1) {
      upd(qv[t], qk[t], base + fx(tab(t)), key);
      if (COUNT) ops += 2 * (nadd + 1);
    }
}

// ---------------------------------------------------------------------------
// closed-interior values Q_t(x, y), every outer type t of the mask tm: the
// loop closed by an outer pair of type t whose interior path runs from x
// (after the 5' nucleotide of the pair) to y (before its 3' nucleotide); x is
// slot sx of layer lx, y slot sy of layer ly.  The options are split into
// classes, and inside a class the G threads of the group take consecutive
// entries of one flat list, so that every thread runs the same inner loops
// (over the out-edges of x and the in-edges of y, the same for the group):
//   hairpin        out-edges of x x in-edges of y (explicit paths for L = 3, 4, 6)
//   stack, bulges  the states of the inner pair's moving end (l1 = 0 or l2 = 0)
//   1 x n          out-edges of the states d of the inner pair (l1 = 1)
//   n x 1          in-edges of the states c of the inner pair (l2 = 1, l1 >= 2)
//   2x2, 2x3, 3x2  (in-edge of c, out-edge of d) pairs
//   generic        out-edges of x x in-edges of y, through the IL table
//   multiloop      one term
// Where the loop energy splits into a part that depends on the inner pair and
// a part that depends on the outer one, the best inner type comes from the
// inner cell's precomputed table W.
// ---------------------------------------------------------------------------
template <int G, bool COUNT>
__device__ __forceinline__ void q_slot(const Fv &F, const SdDesign &D, const SdParams &P,
                                       const SmallTables &T, int sub, int x, int y, int lx,
                                       int sx, int ly, int sy, int tm, int64_t (&qv)[6],
                                       uint32_t (&qk)[6], unsigned long long &ops,
                                       const GapStage &GS) {
  const int g = ly - lx;
  const int nox = F.nout(x), niy = F.nin(y);
  const int lx1s = F.ls(lx + 1), ly1s = F.ls(ly - 1);
  // ---- hairpin (loop length L = g) ----
  if (g == 3 || g == 4 || g == 6) {
    if (sub == 0) {
      // every interior path, lexicographic label order; special loops by sequence
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
#pragma unroll
          for (int t = 0; t < 6; t++)
            if ((tm >> t) & 1) {
              upd(qv[t], qk[t], fx(hairpin_seq_e(P, D.hp_len, t, lb, g)) + cst[g], lb);
              TERM(g);
            }
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
    }
  } else if (g >= 5) {
    const int64_t he = fx(__ldg(&D.hp_len[g]));
    for (int k = sub; k < nox * niy; k += G) {
      const int a = k / niy, b = k - a * niy;
      const SdEdge e1 = F.out(x, a), e2 = F.in(y, b);
      const int64_t h = F.Hh(lx + 1, e1.other - lx1s, ly - 1, e2.other - ly1s);
      if (!fin(h)) continue;
      const int idx = e1.label * 4 + e2.label;
      upd6<COUNT>(qv, qk, tm, e1.cost + e2.cost + h + he, (uint32_t)idx, 3, ops,
                  [&](int t) { return T.mmH[t][idx]; });
    }
  }
  if (g < 5) return;
  // ---- stack and bulges: right side (l1 = 0, l2 = l >= 0), left side (l2 = 0, l1 = l >= 1) ----
  {
    const int rlo = max(ly - SD_MAXTWO, lx + 5);  // layers of d on the right side
    const int r0 = F.ls(rlo), nr = F.ls(ly + 1) - r0;
    const int lhi = min(lx + SD_MAXTWO, ly - 5);  // layers of c on the left side
    const int c0 = lx1s, nl = lhi >= lx + 1 ? F.ls(lhi + 1) - c0 : 0;
    for (int k = sub; k < nr + nl; k += G) {
      const bool right = k < nr;
      const int v = right ? r0 + k : c0 + (k - nr);
      const int lv = F.layer(v), sv = v - F.ls(lv);
      const int l = right ? ly - lv : lv - lx;
      int64_t h = 0;
      int hk = 0;
      if (l > 0) {
        h = right ? GS.hr[l][sv * 2 + sy] : GS.hl[l][sv * 2 + sx];
        if (!fin(h)) continue;
        hk = right ? GS.hrk[l][sv * 2 + sy] : GS.hlk[l][sv * 2 + sx];
      } else if (sv != sy) {
        continue;
      }
      const int cs = right ? sx : sv, ds = right ? sv : sy;
      const uint32_t kb = right ? tl_key(0, l, cs, ds, 0, 0, 0, hk >> 2, hk & 3)
                                : tl_key(l, 0, cs, ds, 0, hk >> 2, hk & 3, 0, 0);
      if (l >= 2) {
        // bulge: bulge[l] + AU(t) + AU(inner); best inner type from the inner table
        const int rc = right ? F.rs(lx, sx, lv, sv) : F.rs(lv, sv, ly, sy);
        const int64_t pk = D.W[(int64_t)rc * SD_WN + 48];
        if (!fin(pk)) continue;
        upd6<COUNT>(qv, qk, tm, (pk >> 3) + h + fx(T.bulge[l]), kb | ((uint32_t)(pk & 7) << 8), 2,
                    ops, [&](int t) { return T.au[t]; });
      } else {
        int64_t vv[6];
        F.v6(right ? F.cs(lx, sx, lv, sv) : F.cs(lv, sv, ly, sy), vv);
        const int64_t e1 = h + fx(l == 1 ? T.bulge[1] : 0);
#pragma unroll
        for (int ti = 0; ti < 6; ti++) {
          if (!fin(vv[ti])) continue;
          const int s = c_rev[ti];
          upd6<COUNT>(qv, qk, tm, vv[ti] + e1, kb | ((uint32_t)ti << 8), 2, ops,
                      [&](int t) { return T.stack[t][s]; });
        }
      }
    }
  }
  // ---- 1 x n: l1 = 1 (nucleotide p after the outer 5' end), l2 >= 1; entries are
  // the out-edges r1 of the inner pair's 3' end d ----
  {
    const int lc = lx + 1;
    const int dlo = max(lx + 6, ly - (SD_MAXTWO - 1)), dhi = ly - 1;
    const int k0 = dlo <= dhi ? F.fo_off[F.ls(dlo)] : 0;
    const int k1 = dlo <= dhi ? F.fo_off[F.ls(dhi + 1)] : 0;
    for (int k = k0 + sub; k < k1; k += G) {
      const SdFlatEdge r1 = F.fo[k];
      const int d = r1.v, u = r1.wl >> 2, fR = r1.wl & 3;
      const int ld = F.layer(d), ds = d - F.ls(ld), l2 = ly - ld;
      if (l2 >= 3) {
        const int lus = F.ls(ld + 1);
        const int64_t e0 = fx(T.interior[1 + l2] + min(T.maxninio, T.ninio * (l2 - 1)));
        for (int a = 0; a < nox; a++) {
          const SdEdge ec = F.out(x, a);
          const int p = ec.label, cs = ec.other - lx1s;
          const int64_t pk = D.W[(int64_t)F.rs(lc, cs, ld, ds) * SD_WN + p * 4 + fR];
          if (!fin(pk)) continue;
          const int64_t base = (pk >> 3) + ec.cost + r1.cost + e0;
          const int wt = (int)(pk & 7);
          for (int b2 = 0; b2 < niy; b2++) {
            const SdEdge r2 = F.in(y, b2);
            const int64_t h = F.Hh(ld + 1, u - lus, ly - 1, r2.other - ly1s);
            if (!fin(h)) continue;
            const int lR = r2.label;
            upd6<COUNT>(qv, qk, tm, base + h + r2.cost, tl_key(1, l2, cs, ds, wt, p, p, fR, lR), 5,
                        ops, [&](int t) { return T.mm1n[t][p * 4 + lR]; });
          }
        }
      } else if (l2 == 1) {
        if (u != y) continue;
        for (int a = 0; a < nox; a++) {
          const SdEdge ec = F.out(x, a);
          const int p = ec.label, cs = ec.other - lx1s;
          int64_t vv[6];
          F.v6(F.cs(lc, cs, ld, ds), vv);
          const int64_t base = ec.cost + r1.cost;
#pragma unroll
          for (int ti = 0; ti < 6; ti++) {
            if (!fin(vv[ti])) continue;
            const int s = c_rev[ti];
            upd6<COUNT>(qv, qk, tm, vv[ti] + base, tl_key(1, 1, cs, ds, ti, p, p, fR, fR), 3, ops,
                        [&](int t) { return P.int11[t][s][p * 4 + fR]; });
          }
        }
      } else {  // l2 == 2: explicit 2-edge right side
        for (int b2 = 0; b2 < F.nout(u); b2++) {
          const SdEdge r2 = F.out(u, b2);
          if (r2.other != y) continue;
          const int lR = r2.label;
          for (int a = 0; a < nox; a++) {
            const SdEdge ec = F.out(x, a);
            const int p = ec.label, cs = ec.other - lx1s;
            int64_t vv[6];
            F.v6(F.cs(lc, cs, ld, ds), vv);
            const int64_t base = ec.cost + r1.cost + r2.cost;
#pragma unroll
            for (int ti = 0; ti < 6; ti++) {
              if (!fin(vv[ti])) continue;
              const int s = c_rev[ti];
              upd6<COUNT>(qv, qk, tm, vv[ti] + base, tl_key(1, 2, cs, ds, ti, p, p, fR, lR), 4,
                          ops, [&](int t) { return P.int21[t][s][p * 16 + fR * 4 + lR]; });
            }
          }
        }
      }
    }
  }
  // ---- n x 1: l2 = 1 (nucleotide r before the outer 3' end), l1 >= 2; entries are
  // the in-edges p2 of the inner pair's 5' end c ----
  {
    const int ld = ly - 1;
    const int clo = lx + 2, chi = min(lx + SD_MAXTWO - 1, ly - 6);
    const int k0 = clo <= chi ? F.fi_off[F.ls(clo)] : 0;
    const int k1 = clo <= chi ? F.fi_off[F.ls(chi + 1)] : 0;
    for (int k = k0 + sub; k < k1; k += G) {
      const SdFlatEdge p2 = F.fi[k];
      const int c = p2.v, w = p2.wl >> 2, lL = p2.wl & 3;
      const int lc = F.layer(c), cs = c - F.ls(lc), l1 = lc - lx;
      if (l1 >= 3) {
        const int lws = F.ls(lc - 1);
        const int64_t e0 = fx(T.interior[l1 + 1] + min(T.maxninio, T.ninio * (l1 - 1)));
        for (int b = 0; b < niy; b++) {
          const SdEdge er = F.in(y, b);
          const int r = er.label, ds = er.other - ly1s;
          const int64_t pk = D.W[(int64_t)F.rs(lc, cs, ld, ds) * SD_WN + lL * 4 + r];
          if (!fin(pk)) continue;
          const int64_t base = (pk >> 3) + er.cost + p2.cost + e0;
          const int wt = (int)(pk & 7);
          for (int a = 0; a < nox; a++) {
            const SdEdge p1 = F.out(x, a);
            const int64_t h = F.Hh(lx + 1, p1.other - lx1s, lc - 1, w - lws);
            if (!fin(h)) continue;
            const int fL = p1.label;
            upd6<COUNT>(qv, qk, tm, base + h + p1.cost, tl_key(l1, 1, cs, ds, wt, fL, lL, r, r), 5,
                        ops, [&](int t) { return T.mm1n[t][fL * 4 + r]; });
          }
        }
      } else {  // l1 == 2: explicit 2-edge left side
        for (int b = 0; b < niy; b++) {
          const SdEdge er = F.in(y, b);
          const int r = er.label, ds = er.other - ly1s;
          int64_t vv[6];
          F.v6(F.cs(lc, cs, ld, ds), vv);
          for (int a = 0; a < nox; a++) {
            const SdEdge p1 = F.out(x, a);
            if (p1.other != w) continue;
            const int fL = p1.label;
            const int64_t base = er.cost + p1.cost + p2.cost;
#pragma unroll
            for (int ti = 0; ti < 6; ti++) {
              if (!fin(vv[ti])) continue;
              const int s = c_rev[ti];
              upd6<COUNT>(qv, qk, tm, vv[ti] + base, tl_key(2, 1, cs, ds, ti, fL, lL, r, r), 4,
                          ops, [&](int t) { return P.int21[s][t][r * 16 + fL * 4 + lL]; });
            }
          }
        }
      }
    }
  }
  // ---- 2x2, 2x3, 3x2: entries are (in-edge p2 of c, out-edge r1 of d) ----
#pragma unroll 1
  for (int cls = 0; cls < 3; cls++) {
    const int l1 = cls == 2 ? 3 : 2, l2 = cls == 1 ? 3 : 2;
    if (g - l1 - l2 < 5) continue;
    const int lc = lx + l1, ld = ly - l2;
    const int lcs = F.ls(lc), lds = F.ls(ld), lc1s = F.ls(lc - 1), ld1s = F.ls(ld + 1);
    const int pi0 = F.fi_off[lcs], npi = F.fi_off[F.ls(lc + 1)] - pi0;
    const int ro0 = F.fo_off[lds], nro = F.fo_off[F.ls(ld + 1)] - ro0;
    for (int k = sub; k < npi * nro; k += G) {
      const int kp = k / nro, kr = k - kp * nro;
      const SdFlatEdge p2 = F.fi[pi0 + kp], r1 = F.fo[ro0 + kr];
      const int cs = p2.v - lcs, ds = r1.v - lds;
      const int w = p2.wl >> 2, lL = p2.wl & 3, u = r1.wl >> 2, fR = r1.wl & 3;
      int64_t vv[6];
      int64_t wv = SD_INF;
      int wt = 7;
      if (cls == 0) {
        F.v6(F.cs(lc, cs, ld, ds), vv);
        if (!(fin(vv[0]) || fin(vv[1]) || fin(vv[2]) || fin(vv[3]) || fin(vv[4]) || fin(vv[5])))
          continue;
      } else {
        const int64_t pk = D.W[(int64_t)F.rs(lc, cs, ld, ds) * SD_WN + 16 + lL * 4 + fR];
        if (!fin(pk)) continue;
        wv = pk >> 3;
        wt = (int)(pk & 7);
      }
      for (int a = 0; a < nox; a++) {
        const SdEdge p1 = F.out(x, a);
        const int64_t hl = F.Hh(lx + 1, p1.other - lx1s, lc - 1, w - lc1s);
        if (!fin(hl)) continue;
        for (int b2 = 0; b2 < niy; b2++) {
          const SdEdge r2 = F.in(y, b2);
          const int64_t hr = F.Hh(ld + 1, u - ld1s, ly - 1, r2.other - ly1s);
          if (!fin(hr)) continue;
          const int64_t hc = p1.cost + p2.cost + r1.cost + r2.cost + hl + hr;
          const int fL = p1.label, lR = r2.label;
          if (cls) {
            upd6<COUNT>(qv, qk, tm, wv + hc + fx(T.interior[5] + T.ninio),
                        tl_key(l1, l2, cs, ds, wt, fL, lL, fR, lR), 8, ops,
                        [&](int t) { return T.mm23[t][fL * 4 + lR]; });
          } else {
            const int idx = fL * 64 + lL * 16 + fR * 4 + lR;
#pragma unroll
            for (int ti = 0; ti < 6; ti++) {
              if (!fin(vv[ti])) continue;
              const int s = c_rev[ti];
              upd6<COUNT>(qv, qk, tm, vv[ti] + hc, tl_key(2, 2, cs, ds, ti, fL, lL, fR, lR), 8,
                          ops, [&](int t) { return P.int22[t][s][idx]; });
            }
          }
        }
      }
    }
  }
  // ---- generic internal loops: mismatch edges + the IL table two spans below ----
  if (g >= 11)
    for (int k = sub; k < nox * niy; k += G) {
      const int a = k / niy, b = k - a * niy;
      const SdEdge e1 = F.out(x, a), e2 = F.in(y, b);
      const int r = F.rs(lx + 1, e1.other - lx1s, ly - 1, e2.other - ly1s);
      const int64_t il = D.IL[r];
      if (!fin(il)) continue;
      const int idx = e1.label * 4 + e2.label;
      upd6<COUNT>(qv, qk, tm, il + e1.cost + e2.cost,
                  (1u << 25) | D.ILk[r] | ((uint32_t)e1.label << 6) | (uint32_t)e2.label, 3, ops,
                  [&](int t) { return T.mmI[t][idx]; });
    }
  // ---- multiloop closed by the pair ----
  if (g >= 10 && sub == G - 1) {
    const int64_t s2 = D.S2[F.cs(lx, sx, ly, sy)];
    if (fin(s2))
      upd6<COUNT>(qv, qk, tm, s2 + fx(T.mlclosing + T.mlintern), KEY_ML, 1, ops,
                  [&](int t) { return T.au[t]; });
  }
}

// (l1', l2') pairs of the generic internal loops, l1'+l2' in [2, 26]
constexpr int IL_PAIRS = 375;

// ---------------------------------------------------------------------------
// the span kernel: a group of G threads (G = 8, 16 or 32) per layer pair
// (i, i+g); consecutive groups take consecutive layer pairs.
// ---------------------------------------------------------------------------
// With G < 32 the groups of one warp take layer pairs i, i+3, i+6, ... (the
// same position inside the codon at both ends, so the same layer types and
// mostly the same branches); a block of 3 warps covers 3 * 32/G consecutive
// layer pairs.
template <int G>
struct FillShape {
  static constexpr int threads = G == 32 ? 128 : 96;
  static constexpr int pairs = threads / G;
  __device__ static int pair_index(int bx) {
    const int warp = (int)threadIdx.x >> 5, grp = ((int)threadIdx.x & 31) / G;
    return G == 32 ? bx * pairs + warp : bx * pairs + warp + 3 * grp;
  }
};


template <int G, bool COUNT>
#ifndef SD_FILL_MINB
#define SD_FILL_MINB 5
#endif
__global__ void __launch_bounds__(FillShape<G>::threads, G == 32 ? 4 : SD_FILL_MINB)
    k_fill_span(const SdDesign *__restrict__ designs, const SdParams *__restrict__ Pp, int g,
                int nact, int items, const int32_t *__restrict__ cpre,
                unsigned long long *ops_out) {
  constexpr int NT = FillShape<G>::threads;
  __shared__ SmallTables T;
  __shared__ uint16_t s_il[IL_PAIRS];
  __shared__ int32_t s_ile[IL_PAIRS];  // size and asymmetry energy of each (l1', l2')
  __shared__ GapStage s_gap[FillShape<G>::pairs];
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
      const int dd = l1p > l2p ? l1p - l2p : l2p - l1p;
      s_ile[r] = Pp->interior[l1p + l2p + 4] + min(Pp->maxninio, Pp->ninio * dd);
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
  F.lay = D.layer;
  F.fo = D.fo;
  F.fo_off = D.fo_off;
  F.fi = D.fi;
  F.fi_off = D.fi_off;
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
  GapStage &GS = s_gap[threadIdx.x / G];
  {
    const int lmax = min(SD_GAPW - 1, g - 1);  // spans below g only (this span is not filled yet)
    for (int q = sub; q < SD_GAPW * 4; q += G) {
      const int l = q >> 2, c = (q >> 1) & 1, sn = q & 1;
      int64_t vl = SD_INF, vr = SD_INF;
      uint8_t kl = 0, kr = 0;
      if (active && l <= lmax) {
        if (sn < wa && c < F.w(i + l)) {
          if (l == 0) {
            vl = c == sn ? 0 : SD_INF;
          } else {
            const int h = F.cs(i, sn, i + l, c);
            vl = F.H[h];
            kl = F.Hk[h];
          }
        }
        if (sn < wb && c < F.w(j - l)) {
          if (l == 0) {
            vr = c == sn ? 0 : SD_INF;
          } else {
            const int h = F.cs(j - l, c, j, sn);
            vr = F.H[h];
            kr = F.Hk[h];
          }
        }
      }
      GS.hl[l][c * 2 + sn] = vl;
      GS.hr[l][c * 2 + sn] = vr;
      GS.hlk[l][c * 2 + sn] = kl;
      GS.hrk[l][c * 2 + sn] = kr;
    }
    __syncwarp();
  }

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
      const int nib = F.nin(b);
#pragma unroll
      for (int k = 0; k < SD_MAXIN; k++) {
        if (k >= nib) break;
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
    // typed closed values (every thread of the group) and Eq. (branch)
    int64_t vv[6];
    {
      const int oma = ok ? D.out_mask[a] : 0, nib = ok ? F.nin(b) : 0;
      const int imb = ok ? D.in_mask[b] : 0;
      int64_t B = SD_INF;
      uint32_t Bk = KEY_NONE;
#pragma unroll
      for (int t = 0; t < 6; t++) {
        int64_t v = SD_INF;
        uint32_t vk = KEY_NONE;
        // the out-edge of a labelled with the pair's 5' nucleotide (a DFA has
        // at most one; out-edges are stored by label)
        const int l5 = c_pair5[t];
        if (ok && g >= 5 && ((oma >> l5) & 1) && ((imb >> c_pair3[t]) & 1)) {
          const SdEdge e1 = F.out(a, __popc(oma & ((1 << l5) - 1)));
          const int l3 = c_pair3[t];
          for (int k2 = 0; k2 < nib; k2++) {
            const SdEdge e2 = F.in(b, k2);
            if (e2.label != l3) continue;
            const int r = F.rs(i + 1, e1.other - i1s, j - 1, e2.other - js) * 6 + t;
            const int64_t q = D.Q[r];
            if (!fin(q)) continue;
            upd(v, vk, q + e1.cost + e2.cost, ((uint32_t)k2 << 27) | D.Qk[r]);
            TERM(2);
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
            best_au(vv, T.au, bv, bt);
          }
        }
        Wc[q] = fin(bv) ? bv * 8 + bt : SD_INF;
      }
    }
  }
  // IL: generic internal loops (l1 = l1'+2, l2 = l2'+2) around every slot of the
  // layer pair at once: each inner cell (c,d) is read once for all slots, the
  // gap values of both ends come from the staged vectors
  if (g >= 9) {
    int64_t lv[SD_SLOTS];
    uint32_t lk[SD_SLOTS];
#pragma unroll
    for (int s = 0; s < SD_SLOTS; s++) {
      lv[s] = SD_INF;
      lk[s] = KEY_NONE;
    }
    if (active)
      for (int q = sub; q < IL_PAIRS; q += G) {
        const int pr = s_il[q];
        const int l1p = pr & 31, l2p = pr >> 5;
        const int lc = i + l1p, ld = j - l2p;
        if (ld - lc < 7) continue;
        const int64_t e = fx(s_ile[q]);
        const uint32_t kl = ((uint32_t)(l1p + l2p + 4) << 20) | ((uint32_t)(l1p + 2) << 15);
        const int rb = (((ld - lc) & (SD_RING - 1)) * (n + 1) + lc) * SD_SLOTS;
        // slots beyond a layer's width have +inf staged gap values
#pragma unroll
        for (int cs = 0; cs < SD_W; cs++) {
          const int64_t hl0 = GS.hl[l1p][cs * 2], hl1 = GS.hl[l1p][cs * 2 + 1];
          if (!fin(hl0) && !fin(hl1)) continue;
#pragma unroll
          for (int ds = 0; ds < SD_W; ds++) {
            const int64_t hr0 = GS.hr[l2p][ds * 2], hr1 = GS.hr[l2p][ds * 2 + 1];
            if (!fin(hr0) && !fin(hr1)) continue;
            const int r = rb + cs * SD_W + ds;
            const int64_t v = D.Ihat[r];
            if (!fin(v)) continue;
            const uint32_t key = kl | D.Ihk[r];
            const int64_t ve = v + e;
#pragma unroll
            for (int s = 0; s < SD_SLOTS; s++) {
              const int64_t h1 = (s >> 1) ? hl1 : hl0, h2 = (s & 1) ? hr1 : hr0;
              if (fin(h1) && fin(h2)) {
                upd(lv[s], lk[s], h1 + ve + h2, key);
                TERM(3);
              }
            }
          }
        }
      }
#pragma unroll
    for (int s = 0; s < SD_SLOTS; s++) {
      seg_lexmin<G>(lv[s], lk[s]);
      settle(lv[s], lk[s]);
      if (active && (s >> 1) < wa && (s & 1) < wb && sub == s % G) {
        D.IL[rcell + s] = lv[s];
        D.ILk[rcell + s] = lk[s];
      }
    }
  } else if (active && sub == 0) {
#pragma unroll
    for (int s = 0; s < SD_SLOTS; s++)
      if ((s >> 1) < wa && (s & 1) < wb) {
        D.IL[rcell + s] = SD_INF;
        D.ILk[rcell + s] = KEY_NONE;
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
        // Eq. (candidates): strict B < P_S; the dense control keeps every
        // finite direct interval (the sparse and dense S2 are equal, Thm. 1)
        if (D.dense ? fin(Bs[s]) : Bs[s] < PSs[s]) {
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
  __syncwarp();  // the stack option reads V of this cell, written by another thread
  // closed-interior values for the pairs two spans up, all outer types at once.
  // The (layer pair, slot) cells that some outer type can close are pooled
  // over the groups of the warp and dealt out round-robin, so that a group
  // with one such cell does not idle while another works through four.
  if constexpr (G == 32) {  // one group per warp: nothing to pool
#pragma unroll 1
    for (int s = 0; s < SD_SLOTS; s++) {
      const int sa = s / SD_W, sb = s % SD_W;
      const bool ok = active && sa < wa && sb < wb;
      int tm = 0;
      if (ok) {
        const int im = D.in_mask[a0 + sa], om = D.out_mask[b0 + sb];
#pragma unroll
        for (int t = 0; t < 6; t++)
          if (((im >> c_pair5[t]) & 1) && ((om >> c_pair3[t]) & 1)) tm |= 1 << t;
      }
      int64_t qv[6];
      uint32_t qk[6];
#pragma unroll
      for (int t = 0; t < 6; t++) {
        qv[t] = SD_INF;
        qk[t] = KEY_NONE;
      }
      if (tm) q_slot<G, COUNT>(F, D, P, T, sub, a0 + sa, b0 + sb, i, sa, j, sb, tm, qv, qk, ops, GS);
#pragma unroll
      for (int t = 0; t < 6; t++) {
        if (tm) seg_lexmin<G>(qv[t], qk[t]);
        settle(qv[t], qk[t]);
        if (ok && sub == t % G) {
          D.Q[(int64_t)(rcell + s) * 6 + t] = qv[t];
          D.Qk[(int64_t)(rcell + s) * 6 + t] = qk[t];
        }
      }
    }
    if (COUNT && active && ops) atomicAdd(&ops_out[dsel], ops);
    return;
  }
  if (COUNT && active && ops) atomicAdd(&ops_out[dsel], ops);
  ops = 0;
  constexpr int NGW = 32 / G;
  const int grp = lane / G;
  uint32_t tms = 0;  // 6 type bits per slot
#pragma unroll
  for (int s = 0; s < SD_SLOTS; s++) {
    const int sa = s / SD_W, sb = s % SD_W;
    const bool ok = active && sa < wa && sb < wb;
    int tm = 0;
    if (ok) {
      const int im = D.in_mask[a0 + sa], om = D.out_mask[b0 + sb];
#pragma unroll
      for (int t = 0; t < 6; t++)
        if (((im >> c_pair5[t]) & 1) && ((om >> c_pair3[t]) & 1)) tm |= 1 << t;
      if (!tm && sub < 6) {  // no outer type can close (x, y)
        D.Q[(int64_t)(rcell + s) * 6 + sub] = SD_INF;
        D.Qk[(int64_t)(rcell + s) * 6 + sub] = KEY_NONE;
      }
    }
    tms |= (uint32_t)tm << (6 * s);
  }
  uint32_t words[NGW];
  int K = 0;
#pragma unroll
  for (int go = 0; go < NGW; go++) {
    words[go] = __shfl_sync(FULL, tms, go * G);
#pragma unroll
    for (int s = 0; s < SD_SLOTS; s++) K += ((words[go] >> (6 * s)) & 63) != 0;
  }
#pragma unroll 1
  for (int r = 0; r < K; r += NGW) {
    // this group's cell of the round: the (r + grp)-th pooled one
    const int k = r + grp;
    int go_k = 0, s_k = 0, tm_k = 0, c = 0;
#pragma unroll
    for (int go = 0; go < NGW; go++)
#pragma unroll
      for (int s = 0; s < SD_SLOTS; s++) {
        const int tmv = (words[go] >> (6 * s)) & 63;
        if (tmv) {
          if (c == k) {
            go_k = go;
            s_k = s;
            tm_k = tmv;
          }
          c++;
        }
      }
    const int src = go_k * G;
    const int o_dsel = __shfl_sync(FULL, dsel, src), o_i = __shfl_sync(FULL, i, src);
    const int o_a0 = __shfl_sync(FULL, a0, src), o_b0 = __shfl_sync(FULL, b0, src);
    int64_t qv[6];
    uint32_t qk[6];
#pragma unroll
    for (int t = 0; t < 6; t++) {
      qv[t] = SD_INF;
      qk[t] = KEY_NONE;
    }
    const SdDesign &Do = designs[o_dsel];
    const int sa = s_k / SD_W, sb = s_k % SD_W;
    if (tm_k) {
      Fv Fo;
      Fo.n = Do.n;
      Fo.lst = Do.lstart;
      Fo.oe = Do.out;
      Fo.ie = Do.in;
      Fo.on = Do.out_cnt;
      Fo.in_ = Do.in_cnt;
      Fo.H = Do.H;
      Fo.Hk = Do.Hk;
      Fo.V = Do.V;
      Fo.lay = Do.layer;
      Fo.fo = Do.fo;
      Fo.fo_off = Do.fo_off;
      Fo.fi = Do.fi;
      Fo.fi_off = Do.fi_off;
      q_slot<G, COUNT>(Fo, Do, P, T, sub, o_a0 + sa, o_b0 + sb, o_i, sa, o_i + g, sb, tm_k, qv,
                       qk, ops, s_gap[(threadIdx.x >> 5) * NGW + go_k]);
    }
    const int o_rcell = ((g & (SD_RING - 1)) * (Do.n + 1) + o_i) * SD_SLOTS;
#pragma unroll
    for (int t = 0; t < 6; t++) {
      if (__any_sync(FULL, (tm_k >> t) & 1)) seg_lexmin<G>(qv[t], qk[t]);
      settle(qv[t], qk[t]);
      if (tm_k && sub == t % G) {
        Do.Q[(int64_t)(o_rcell + s_k) * 6 + t] = qv[t];
        Do.Qk[(int64_t)(o_rcell + s_k) * 6 + t] = qk[t];
      }
    }
    if (COUNT && tm_k && ops) atomicAdd(&ops_out[o_dsel], ops);
    ops = 0;
  }
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
  constexpr int per_block = FillShape<G>::pairs;
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
    case 8: launch_fill_g<8, COUNT>(d_designs, count, ns, d_cpre, d_params, st, d_ops); break;
    case 16: launch_fill_g<16, COUNT>(d_designs, count, ns, d_cpre, d_params, st, d_ops); break;
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

// An event record that also becomes an event-record node when the stream is
// being captured into a graph (a plain record there is only a capture
// dependency and would not fire when the graph is replayed).
static void record(void *ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags((cudaEvent_t)ev, st, cudaEventRecordExternal);
  else
    cudaEventRecord((cudaEvent_t)ev, st);
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
  if (events) record(events[0], st);
  if (launch_fill<false>(group, d_designs, count, ns, d_cpre, d_params, st, nullptr)) return -1;
  if (events) record(events[1], st);
  k_exterior<<<count, 256, 0, st>>>(d_designs, d_params);
  if (events) record(events[2], st);
  k_traceback<<<count, 128, 0, st>>>(d_designs, d_params);
  if (events) record(events[3], st);
  if (launches) *launches = (int64_t)ns[0] + 3;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
