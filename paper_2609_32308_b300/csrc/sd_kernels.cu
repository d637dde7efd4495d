// sd_kernels.cu -- sm_103a kernels of the exact codon-lattice design DP.
//
// Span wavefront (Algorithm 1, Sec. 5).  One launch per span g processes every
// layer pair (i, i+g) of every design in the batch (a work queue over
// (design, layer pair), longest design first), one group of 8, 16 or 32
// threads per layer pair.  The paper separates closed/gap values, multiloop
// values and exterior values by barriers; here all phases of one layer pair run
// in the group that owns it, because each only reads smaller spans or the same
// cell:
//   stage  gap vectors of both ends (mirrors GL / GR)            spans 0..30 (< g)
//   H      min path cost a->b (gap cells)                       span g-1
//   Ihat   inner pair + its loop-side mismatch (two-loop inner)  V at span g-2
//   V_t    typed closed value (Sec. 4.1)                         Q at span g-2
//   B, WB  Eq. (branch); the bulge term of the cell              V of this cell
//   X, Y   one-nucleotide-side factors of 1 x n / n x 1 loops    V at span g-1
//   Af     two-loop factors (1 x n, n x 1, 2x3, 3x2)             X / Y windows, V
//   IL, K  generic internal loops by loop size                   Ihat spans g..g-26, K at g-2
//   S2     Eq. (sparse2): edge extension + candidate splits      spans < g
//   S1     P_S, S1 = min(B, P_S), strict test B < P_S (Eq. candidates)
//   Q_t    hairpin / two-loop / multiloop interior for outer type t (read by V at g+2)
// The owner of layer pair (i, i+g) is the only writer of C_b for b on layer
// i+g at span g (Sec. 5 endpoint ownership), and it scans C_b before it
// appends, so no lock or barrier is needed inside a span.
//
// Values only.  The fill stores the minimum of every cell and nothing about
// which option attains it: a minimum does not depend on the order in which
// the options are visited, so the fill is free to visit them in whatever
// order suits the hardware.  The canonical choice of every traced cell (the
// first attaining option of a fixed enumeration, Sec. 4.2 leaves ties open)
// is re-derived afterwards by the traceback from the full tables.
//
// The exterior (final-column) values and the traceback run after the fill,
// one 1,024-thread block per design.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sd_internal.h"

// The host entry points of this file; the wide instance (SD_W > 2, compiled
// from sd_kernels_wide.cu) carries the suffix _wide.
#if SD_W == 2
#define SD_KFN(name) name
#else
#define SD_KFN(name) name##_wide
#endif

static_assert(SD_W <= (1 << SD_CAND_SHIFT), "a candidate entry holds the slot in SD_CAND_SHIFT bits");

namespace {

constexpr unsigned FULL = 0xffffffffu;

__constant__ int c_pair5[6] = {0, 1, 2, 3, 2, 3};
__constant__ int c_pair3[6] = {3, 2, 1, 0, 3, 2};

__device__ __forceinline__ int64_t fx(int e) { return (int64_t)e * 4294967296LL; }

// Reads of cells filled by earlier launches (every span below the current
// one) go through the read-only data path; cells of the current span (the
// stack option's inner cell, the multiloop option's S2) are read coherently.
#ifndef SD_NC
#define SD_NC 1
#endif
template <class T>
__device__ __forceinline__ T ro(const T *p) {
#if SD_NC
  return __ldg(p);
#else
  return *p;
#endif
}
__device__ __forceinline__ bool fin(int64_t v) { return v < SD_FINLIM; }

__device__ __forceinline__ int64_t diag_off(int64_t n, int64_t g) {
  return (g - 1) * (n + 1) - (g - 1) * g / 2;
}

__device__ __forceinline__ void upd(int64_t &bv, int64_t v) { bv = v < bv ? v : bv; }
__device__ __forceinline__ void warp_min(int64_t &v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) upd(v, __shfl_xor_sync(FULL, v, o));
}
// every value >= 2^59 is +infinity; store it as SD_INF
__device__ __forceinline__ int64_t settle(int64_t v) { return fin(v) ? v : SD_INF; }

struct Lat {
  const SdDesign &D;
  __device__ Lat(const SdDesign &d) : D(d) {}
  __device__ __forceinline__ int layer(int v) const { return __ldg(&D.layer[v]); }
  __device__ __forceinline__ int lstart(int l) const { return __ldg(&D.lstart[l]); }
  // entry of state pair (x, y), x on layer lx, y on a later layer ly
  __device__ __forceinline__ int64_t slot(int x, int y, int lx, int ly) const {
    if (D.layout == SD_LAYOUT_SQUARE) return (int64_t)x * D.N + y;
    if (D.layout == SD_LAYOUT_PACKED) return __ldg(&D.poff[x]) + (y - lstart(lx + 1));
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
  __device__ __forceinline__ SdEdge in(int v, int k) const { return D.in[v * D.maxin + k]; }
  __device__ __forceinline__ int out_with_label(int v, int lab) const {
    for (int k = 0; k < nout(v); k++)
      if (D.out[v * SD_MAXOUT + k].label == lab) return k;
    return -1;
  }
};

// ---------------------------------------------------------------------------
// loop energies (integer dcal/mol), Sec. 3 model
// ---------------------------------------------------------------------------

__device__ __forceinline__ int hairpin_generic_e(const SdParams &P, const int32_t *hp_len, int t,
                                                 int L, int f, int l) {
  if (L == 3) return __ldg(&hp_len[3]) + P.au[t];
  return __ldg(&hp_len[L]) + P.mmH[t][f * 4 + l];
}

// hairpin energy of the complete hairpin: pair t, loop labels packed 2 bits
// each with the first loop label most significant
__device__ __noinline__ int hairpin_seq_e(const SdParams &P, const int32_t *hp_len, int t,
                                          uint32_t labs, int L) {
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
__device__ __forceinline__ void seg_min(int64_t &v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) upd(v, __shfl_xor_sync(FULL, v, o));
}

// Minimum of eight values across the G >= 8 threads of a group, each thread
// ending with one of them: recursive halving (every exchange step trades half
// of the values still held), so the result of value (sub & 7) lands in thread
// sub after 4 + 2 + 1 exchanges instead of 8 * log2(G).
template <int G>
__device__ __forceinline__ int64_t seg_min8(const int64_t *x, int sub) {
  const bool b2 = (sub >> 2) & 1, b1 = (sub >> 1) & 1, b0 = sub & 1;
  int64_t y[4], z[2];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const int64_t r = __shfl_xor_sync(FULL, b2 ? x[k] : x[k + 4], 4);
    y[k] = b2 ? x[k + 4] : x[k];
    upd(y[k], r);
  }
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const int64_t r = __shfl_xor_sync(FULL, b1 ? y[k] : y[k + 2], 2);
    z[k] = b1 ? y[k + 2] : y[k];
    upd(z[k], r);
  }
  int64_t v = b0 ? z[1] : z[0];
  upd(v, __shfl_xor_sync(FULL, b0 ? z[0] : z[1], 1));
#pragma unroll
  for (int o = 8; o < G; o <<= 1) upd(v, __shfl_xor_sync(FULL, v, o));
  return v;
}

// Design view for the fill: hot pointers in registers, 32-bit index math
// (sizes are limited to n <= 12000 nucleotides on the host).
struct Fv {
  int n, N, layout, maxin;
  const int64_t *__restrict__ poff;
  const int32_t *__restrict__ lst;
  const SdEdge *__restrict__ oe;
  const SdEdge *__restrict__ ie;
  const uint8_t *__restrict__ on;
  const uint8_t *__restrict__ in_;
  const int64_t *H;
  const int64_t *V;
  const SdFlatEdge *__restrict__ fo;
  const int32_t *__restrict__ fo_off;
  const SdFlatEdge *__restrict__ fi;
  const int32_t *__restrict__ fi_off;
  __device__ __forceinline__ int ls(int l) const { return __ldg(lst + l); }
  __device__ __forceinline__ int w(int l) const { return __ldg(lst + l + 1) - __ldg(lst + l); }
  __device__ __forceinline__ int doff(int s) const { return (s - 1) * (n + 1) - (((s - 1) * s) >> 1); }
  // full-table entry of (layer lx, slot sx) -> (layer ly, slot sy), ly > lx
  __device__ __forceinline__ int cs(int lx, int sx, int ly, int sy) const {
    if (layout == SD_LAYOUT_SPAN) return (doff(ly - lx) + lx) * SD_SLOTS + sx * SD_W + sy;
    const int a = ls(lx) + sx;
    if (layout == SD_LAYOUT_SQUARE) return a * N + ls(ly) + sy;
    return (int)(__ldg(poff + a) + (ls(ly) + sy - ls(lx + 1)));
  }
  __device__ __forceinline__ int rs(int lx, int sx, int ly, int sy) const {
    return (((ly - lx) & (SD_RING - 1)) * (n + 1) + lx) * SD_SLOTS + sx * SD_W + sy;
  }
  // min path cost, 0 on the same state, +inf on another state of the same layer
  __device__ __forceinline__ int64_t Hh(int lx, int sx, int ly, int sy) const {
    if (ly == lx) return sx == sy ? 0 : SD_INF;
    return ro(H + cs(lx, sx, ly, sy));
  }
  __device__ __forceinline__ int nout(int v) const { return on[v]; }
  __device__ __forceinline__ int nin(int v) const { return in_[v]; }
  __device__ __forceinline__ SdEdge out(int v, int k) const { return oe[v * SD_MAXOUT + k]; }
  __device__ __forceinline__ SdEdge in(int v, int k) const { return ie[v * maxin + k]; }
  // V of a cell of an earlier span (read-only path)
  __device__ __forceinline__ void v6(int idx, int64_t (&vv)[6]) const {
    const longlong2 *p = reinterpret_cast<const longlong2 *>(V + (int64_t)idx * 6);
    const longlong2 a = ro(p), b = ro(p + 1), c = ro(p + 2);
    vv[0] = a.x;
    vv[1] = a.y;
    vv[2] = b.x;
    vv[3] = b.y;
    vv[4] = c.x;
    vv[5] = c.y;
  }
};

// Gap values of the two ends of a layer pair: hl[l][c*W + s] = H(slot s of
// layer i -> slot c of layer i+l), hr[l][c*W + s] = H(slot c of layer j-l ->
// slot s of layer j), l < SD_GAPW; the two-loop options read them many
// times.  Narrow layers stage them in shared memory per group; wide layers
// (64 slots, 31 KB per layer pair) read the gap mirrors in global memory, so
// that more groups fit on an SM.
struct alignas(16) GapStage {
  int64_t hl[SD_W == 2 ? SD_GAPW : 1][SD_SLOTS], hr[SD_W == 2 ? SD_GAPW : 1][SD_SLOTS];
};
struct GapRows {
  const int64_t (*hl)[SD_SLOTS];
  const int64_t (*hr)[SD_SLOTS];
};

// A V row of an earlier span (read-only path), or of this span: the values
// and the mask of the finite types (bit t for a finite V_t).  The type loops
// then visit the finite types only (most pairs admit one or two), picking
// each value by constant-index selects.
template <bool CUR>
__device__ __forceinline__ int vrow(const int64_t *vr, int64_t (&v)[6]) {
  const longlong2 *p = reinterpret_cast<const longlong2 *>(vr);
  const longlong2 a = CUR ? p[0] : ro(p), b = CUR ? p[1] : ro(p + 1), c = CUR ? p[2] : ro(p + 2);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
  v[4] = c.x;
  v[5] = c.y;
  int fm = 0;
#pragma unroll
  for (int t = 0; t < 6; t++) fm |= (int)fin(v[t]) << t;
  return fm;
}
__device__ __forceinline__ int64_t pick6(const int64_t (&v)[6], int t) {
  int64_t r = v[0];
#pragma unroll
  for (int q = 1; q < 6; q++)
    if (t == q) r = v[q];
  return r;
}

// the type of the same pair read from the other strand (AU <-> UA, CG <-> GC,
// GU <-> UG)
__device__ __forceinline__ int rev_type(int t) { return t < 4 ? 3 - t : 9 - t; }

// minimum over the inner pair types of vv[ti] + tab[rev ti][idx] (the finite
// types only)
__device__ __forceinline__ int64_t best_inner(const int64_t (&vv)[6], const int32_t (*tab)[16],
                                              int idx) {
  int fm = 0;
#pragma unroll
  for (int t = 0; t < 6; t++) fm |= (int)fin(vv[t]) << t;
  int64_t bv = SD_INF;
  for (; fm; fm &= fm - 1) {
    const int ti = __ffs(fm) - 1;
    upd(bv, pick6(vv, ti) + fx(tab[rev_type(ti)][idx]));
  }
  return bv;
}

// All outer pair types of one closed-interior cell at once: qv[t] is the
// running minimum of Q_t for every t in the type mask tm (the same for every
// thread of a group).  tab(t) is the outer-type part of the loop energy; the
// rest of the term is shared by the types.
template <bool COUNT, class Tab>
__device__ __forceinline__ void upd6(int64_t (&qv)[6], int tm, int64_t base, int nadd,
                                     unsigned long long &ops, const Tab &tab) {
#pragma unroll
  for (int t = 0; t < 6; t++)
    if ((tm >> t) & 1) {
      upd(qv[t], base + fx(tab(t)));
      if (COUNT) ops += 2 * (nadd + 1);
    }
}

// ---------------------------------------------------------------------------
// closed-interior values Q_t(x, y), every outer type t of the mask tm: the
// loop closed by an outer pair of type t whose interior path runs from x
// (after the 5' nucleotide of the pair) to y (before its 3' nucleotide); x is
// slot sx of layer lx, y slot sy of layer ly.  The options are split into
// classes, and inside a class the G threads of the group take consecutive
// entries of one list:
//   hairpin           out-edges of x x in-edges of y (explicit paths for L = 3, 4, 6)
//   stack, bulges     the states of the inner pair's moving end (l1 = 0 or l2 = 0);
//                     bulges l >= 2 take the inner cell's bulge term WB
//   1 x 1, 1 x 2      the one- and two-edge right sides into y
//   2 x 1, 2 x 2      the two-edge left sides out of x, each with the right sides
//   generic, 1 x n, n x 1 (long side >= 3), 2x3, 3x2
//                     out-edges of x x in-edges of y, through the tables IL and Af
//                     of the cell one nucleotide inside
//   multiloop         one term
// ---------------------------------------------------------------------------
template <int G, bool COUNT>
__device__ __forceinline__ void q_slot(const Fv &F, const SdDesign &D, const SdParams &P,
                                       const SmallTables &T, int sub, int x, int y, int lx,
                                       int sx, int ly, int sy, int tm, int64_t (&qv)[6],
                                       unsigned long long &ops, const GapRows &GS) {
  const int g = ly - lx;
  const int nox = F.nout(x), niy = F.nin(y);
  // (the 1x1 / 1x2 tables stay in global memory: a larger shared-memory
  // carve-out would cost this kernel its L1 hit rate)
  const int32_t(*I11)[6][16] = P.int11;
  const int32_t(*I21)[6][64] = P.int21;
  const int lx1s = F.ls(lx + 1), ly1s = F.ls(ly - 1);
  // ---- hairpin (loop length L = g) ----
  if (g == 3 || g == 4 || g == 6) {
    if (sub == 0) {
      // every interior path; special loops by sequence
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
              upd(qv[t], fx(hairpin_seq_e(P, D.hp_len, t, lb, g)) + cst[g]);
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
#pragma unroll 1
    for (int k = sub; k < nox * niy; k += G) {
      const int a = k / niy, b = k - a * niy;
      const SdEdge e1 = F.out(x, a), e2 = F.in(y, b);
      const int64_t h = F.Hh(lx + 1, e1.other - lx1s, ly - 1, e2.other - ly1s);
      if (!fin(h)) continue;
      const int idx = e1.label * 4 + e2.label;
      upd6<COUNT>(qv, tm, e1.cost + e2.cost + h + he, 3, ops, [&](int t) { return T.mmH[t][idx]; });
    }
  }
  if (g < 5) return;
  // ---- stack and bulges: right side (l1 = 0, l2 = l >= 0), left side (l2 = 0, l1 = l >= 1) ----
  {
    // the states d of the right side, c of the left side
    const int r0 = F.ls(max(ly - SD_MAXTWO, lx + 5)), nr = F.ls(ly + 1) - r0;
    const int lhi = min(lx + SD_MAXTWO, ly - 5);
    const int nl = lhi >= lx + 1 ? F.ls(lhi + 1) - lx1s : 0;
    int64_t bul = SD_INF;  // bulges l >= 2: inner part, AU(t) added once below
#pragma unroll 1
    for (int k = sub; k < nr + nl; k += G) {
      const bool right = k < nr;
      const int pv = __ldg(&D.pos[right ? r0 + k : lx1s + k - nr]);
      const int lv = pv >> SD_CAND_SHIFT, sv = pv & ((1 << SD_CAND_SHIFT) - 1);
      const int l = right ? ly - lv : lv - lx;
      // staged gap (l = 0: 0 on y itself, +inf elsewhere)
      const int64_t h = right ? GS.hr[l][sv * SD_W + sy] : GS.hl[l][sv * SD_W + sx];
      if (!fin(h)) continue;
      if (l >= 2) {
        // bulge: bulge[l] + AU(t) + AU(inner); best inner type from WB
        const int rc = right ? F.rs(lx, sx, lv, sv) : F.rs(lv, sv, ly, sy);
        const int64_t w = ro(D.WB + rc);
        if (!fin(w)) continue;
        upd(bul, w + h + fx(T.bulge[l]));
        TERM(2);
      } else {
        const int vc = right ? F.cs(lx, sx, lv, sv) : F.cs(lv, sv, ly, sy);
        const int64_t *vr = F.V + (int64_t)vc * 6;
        const int64_t e1 = h + fx(l == 1 ? T.bulge[1] : 0);
        int64_t vv[6];
        for (int fm = l == 0 ? vrow<true>(vr, vv) : vrow<false>(vr, vv); fm; fm &= fm - 1) {
          const int ti = __ffs(fm) - 1, s = rev_type(ti);
          upd6<COUNT>(qv, tm, pick6(vv, ti) + e1, 2, ops, [&](int t) { return T.stack[t][s]; });
        }
      }
    }
    if (fin(bul)) upd6<COUNT>(qv, tm, bul, 0, ops, [&](int t) { return T.au[t]; });
  }
  // ---- 1 x 1 and 1 x 2: l1 = 1 (nucleotide p after the outer 5' end), l2 <= 2
  // (1 x n with l2 >= 3 comes from the factor table Af below).  Entries: the
  // in-edges r1: d -> y (l2 = 1), then the in-edges r2: u -> y, each with the
  // in-edges r1: d -> u of its source (l2 = 2); the inner pair (c, d) needs
  // d at least 5 layers after c ----
  {
    const int lc = lx + 1;
    const int n1 = ly - 1 >= lx + 6 ? niy : 0, n2 = ly - 2 >= lx + 6 ? niy : 0;
    const int ly2s = F.ls(ly - 2);
#pragma unroll 1
    for (int k = sub; k < n1 + n2; k += G) {
      const bool one = k < n1;  // l2 = 1
      const SdEdge er = F.in(y, one ? k : k - n1);
      // l2 = 1: er is r1 (d = its source); l2 = 2: er is r2 (u = its source)
      const int nr1 = one ? 1 : F.nin(er.other);
#pragma unroll 1
      for (int k1 = 0; k1 < nr1; k1++) {
        const SdEdge r1 = one ? er : F.in(er.other, k1);
        const int ds = r1.other - (one ? ly1s : ly2s), fR = r1.label;
        const int64_t rc = one ? r1.cost : r1.cost + er.cost;
        const int idx2 = fR * 4 + er.label;  // 1 x 2: (fR, lR)
#pragma unroll 1
        for (int a = 0; a < nox; a++) {
          const SdEdge ec = F.out(x, a);
          const int p = ec.label, cs = ec.other - lx1s;
          const int64_t *vr = F.V + (int64_t)F.cs(lc, cs, one ? ly - 1 : ly - 2, ds) * 6;
          const int64_t base = ec.cost + rc;
          int64_t vv[6];
          for (int fm = vrow<false>(vr, vv); fm; fm &= fm - 1) {
            const int ti = __ffs(fm) - 1, s = rev_type(ti);
            const int64_t v = pick6(vv, ti);
            if (one)
              upd6<COUNT>(qv, tm, v + base, 3, ops, [&](int t) { return I11[t][s][p * 4 + fR]; });
            else
              upd6<COUNT>(qv, tm, v + base, 4, ops,
                          [&](int t) { return I21[t][s][p * 16 + idx2]; });
          }
        }
      }
    }
  }
  // ---- 2 x 1 (l1 = 2, l2 = 1) and 2 x 2 (l1 = l2 = 2): the entries are the
  // two-edge left sides x -> w -> c (p1, p2), by (p1, out-edge slot of w);
  // each takes the right sides into y: the in-edges r: d -> y (2 x 1), and
  // the in-edges r2: u -> y with the in-edges r1: d -> u of u (2 x 2)
  // (2x3 and 3x2 come from Af) ----
  if (g >= 8) {
    const int lc = lx + 2, lcs = F.ls(lc), ly2s = F.ls(ly - 2);
#pragma unroll 1
    for (int k = sub; k < nox * SD_MAXOUT; k += G) {
      const SdEdge p1 = F.out(x, k / SD_MAXOUT);
      const int b = k % SD_MAXOUT;
      if (b >= F.nout(p1.other)) continue;
      const SdEdge p2 = F.out(p1.other, b);
      const int cs = p2.other - lcs, fL = p1.label, lL = p2.label;
      const int64_t lcost = p1.cost + p2.cost;
#pragma unroll 1
      for (int b2 = 0; b2 < niy; b2++) {
        const SdEdge er = F.in(y, b2);
        // 2 x 1: d = the source of er, on layer ly - 1
        {
          const int64_t *vr = F.V + (int64_t)F.cs(lc, cs, ly - 1, er.other - ly1s) * 6;
          const int64_t base = er.cost + lcost;
          const int r = er.label;
          int64_t vv[6];
          for (int fm = vrow<false>(vr, vv); fm; fm &= fm - 1) {
            const int ti = __ffs(fm) - 1, s = rev_type(ti);
            upd6<COUNT>(qv, tm, pick6(vv, ti) + base, 4, ops,
                        [&](int t) { return I21[s][t][r * 16 + fL * 4 + lL]; });
          }
        }
        // 2 x 2: er is r2 (u = its source), d -> u on layer ly - 2
        if (g >= 9) {
          const int u = er.other;
#pragma unroll 1
          for (int b1 = 0; b1 < F.nin(u); b1++) {
            const SdEdge r1 = F.in(u, b1);
            const int64_t *vr = F.V + (int64_t)F.cs(lc, cs, ly - 2, r1.other - ly2s) * 6;
            const int64_t hc = lcost + r1.cost + er.cost;
            const int idx = fL * 64 + lL * 16 + r1.label * 4 + er.label;
            int64_t vv[6];
            for (int fm = vrow<false>(vr, vv); fm; fm &= fm - 1) {
              const int ti = __ffs(fm) - 1, s = rev_type(ti);
              upd6<COUNT>(qv, tm, pick6(vv, ti) + hc, 8, ops, [&](int t) { return P.int22[t][s][idx]; });
            }
          }
        }
      }
    }
  }
  // ---- loops reached through the cell one nucleotide inside (c, d): the outer
  // mismatch edges e1 = x -> c (label p), e2 = d -> y (label r) plus the
  // cell's tables two spans below: generic internal loops (IL), 1 x n and n x 1
  // with the long side >= 3 and 2x3 / 3x2 (the factors Af) ----
  if (g >= 9)
#pragma unroll 1
    for (int k = sub; k < nox * niy; k += G) {
      const int a = k / niy, b = k - a * niy;
      const SdEdge e1 = F.out(x, a), e2 = F.in(y, b);
      const int r = F.rs(lx + 1, e1.other - lx1s, ly - 1, e2.other - ly1s);
      const int idx = e1.label * 4 + e2.label;
      const int64_t base = e1.cost + e2.cost;
      if (g >= 11) {
        const int64_t il = ro(D.IL + r);
        if (fin(il)) upd6<COUNT>(qv, tm, il + base, 3, ops, [&](int t) { return T.mmI[t][idx]; });
      }
      const int64_t *af = D.Af + (int64_t)r * SD_AN;
      const int64_t a1 = ro(af + e1.label), a2 = ro(af + 4 + e2.label);
      const int64_t m1 = a1 < a2 ? a1 : a2;
      if (fin(m1)) upd6<COUNT>(qv, tm, m1 + base, 3, ops, [&](int t) { return T.mm1n[t][idx]; });
      const int64_t a23 = ro(af + 8);
      if (fin(a23)) upd6<COUNT>(qv, tm, a23 + base, 3, ops, [&](int t) { return T.mm23[t][idx]; });
    }
  // ---- multiloop closed by the pair ----
  if (g >= 10 && sub == G - 1) {
    const int64_t s2 = D.S2[F.cs(lx, sx, ly, sy)];
    if (fin(s2))
      upd6<COUNT>(qv, tm, s2 + fx(T.mlclosing + T.mlintern), 1, ops,
                  [&](int t) { return T.au[t]; });
  }
}


// ---------------------------------------------------------------------------
// the span kernel: a group of G threads (G = 8, 16 or 32) per layer pair
// (i, i+g); consecutive groups take consecutive layer pairs.
// ---------------------------------------------------------------------------
// With G < 32 the groups of one warp take layer pairs i, i+3, i+6, ... (the
// same position inside the codon at both ends, so the same layer types and
// mostly the same branches); a block of 3 warps covers 3 * 32/G consecutive
// layer pairs.

#ifndef SD_FILL_WARPS
#define SD_FILL_WARPS 3  // warps per block for groups of 8 or 16 (a multiple of 3)
#endif
template <int G>
struct FillShape {
  // wide layers (SD_W > 2) stage large gap vectors: one group per block
  static constexpr int threads = G == 32 ? (SD_W > 2 ? 32 : 128) : 32 * SD_FILL_WARPS;
  static constexpr int pairs = threads / G;
  __device__ static int pair_index(int bx) {
    const int warp = (int)threadIdx.x >> 5, grp = ((int)threadIdx.x & 31) / G;
    return G == 32 ? bx * pairs + warp
                   : bx * pairs + warp % 3 + 3 * (grp + (32 / G) * (warp / 3));
  }
};


// Bulk copy of one row of a gap mirror into shared memory (16-byte aligned
// addresses, a multiple of 16 bytes), completing on the group's barrier.
constexpr uint32_t SD_GAP_ROW = SD_GAPW * SD_SLOTS * 8;
static_assert(SD_GAP_ROW % 16 == 0, "bulk copies move multiples of 16 bytes");
__device__ __forceinline__ void bulk_row(uint32_t dst, const int64_t *src, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(SD_GAP_ROW), "r"(bar)
      : "memory");
}
// Wait for phase 0 of a transaction barrier for at most ~1 s of SM clock.
__device__ __forceinline__ bool wait_phase0(uint32_t bar) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
        " selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(bar) : "memory");
    if (done) return true;
    if (clock64() - t0 > (1LL << 31)) return false;
  }
}
// Stage the group's two gap rows; false when some group's copies in the warp
// did not complete in time (every design of the warp's layer pairs is flagged
// invalid and the warp leaves).
__device__ __forceinline__ bool stage_gap_rows(const SdDesign &D, bool active, int sub, int i,
                                               int j, GapStage &GS, uint64_t &barw) {
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&barw);
  if (active && sub == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"(2 * SD_GAP_ROW)
                 : "memory");
    bulk_row((uint32_t)__cvta_generic_to_shared(&GS.hl[0][0]),
             D.GL + (int64_t)i * SD_GAPW * SD_SLOTS, bar);
    bulk_row((uint32_t)__cvta_generic_to_shared(&GS.hr[0][0]),
             D.GR + (int64_t)j * SD_GAPW * SD_SLOTS, bar);
  }
  __syncwarp();
  const bool late = active && !wait_phase0(bar);
  if (__any_sync(FULL, late)) {
    if (active && sub == 0) {
      // this layer pair stays unfilled
      atomicOr(reinterpret_cast<unsigned long long *>(&D.tb[3]), (unsigned long long)SD_TB_WAIT);
      if (late) wait_phase0(bar);  // the copies may still be in flight into this block's memory
    }
    __syncwarp();
    return false;
  }
  return true;
}

#ifndef SD_FILL_MINB
#define SD_FILL_MINB 5
#endif
template <int G, bool COUNT>
__global__ void __launch_bounds__(FillShape<G>::threads, G == 32 ? 4 : SD_FILL_MINB)
    k_fill_span(const SdDesign *__restrict__ designs, const SdParams *__restrict__ Pp, int g,
                int nact, int items, const int32_t *__restrict__ cpre,
                unsigned long long *ops_out) {
  constexpr int NT = FillShape<G>::threads;
  __shared__ SmallTables T;
  __shared__ GapStage s_gap[FillShape<G>::pairs];
  __shared__ uint64_t s_bar[FillShape<G>::pairs];  // one transaction barrier per group
  {
    const int32_t *src[] = {&Pp->stack[0][0], &Pp->mmH[0][0], &Pp->bulge[0], &Pp->au[0],
                            &Pp->ninio};
    int32_t *dst[] = {&T.stack[0][0], &T.mmH[0][0], &T.bulge[0], &T.au[0], &T.ninio};
    const int cnt[] = {36, 4 * 96, 64, 6, 5};
#pragma unroll
    for (int q = 0; q < 5; q++)
      for (int k = threadIdx.x; k < cnt[q]; k += NT) dst[q][k] = src[q][k];
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
  F.N = D.N;
  F.layout = D.layout;
  F.maxin = D.maxin;
  F.poff = D.poff;
  F.lst = D.lstart;
  F.oe = D.out;
  F.ie = D.in;
  F.on = D.out_cnt;
  F.in_ = D.in_cnt;
  F.H = D.H;
  F.V = D.V;
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
  const int rcell = ((g & (SD_RING - 1)) * (n + 1) + i) * SD_SLOTS;
  const int64_t mlb = fx(T.mlbase);
  const int js = active ? F.ls(j - 1) : 0;  // first state on layer j-1
  const int i1s = active ? F.ls(i + 1) : 0;
  GapStage &GSt = s_gap[threadIdx.x / G];
  // The gap mirrors of layer i (from the left) and layer j (from the right),
  // one contiguous row each, copied into the group's stage by two bulk
  // asynchronous copies that one thread issues and a transaction barrier
  // tracks.  Entries of spans >= g still hold the +inf of the run's reset (the
  // mirrors of span l are written by the launch of span l).
  GapRows GS;
  if constexpr (SD_W == 2) {
    if (!stage_gap_rows(D, active, sub, i, j, GSt, s_bar[threadIdx.x / G])) return;
    GS = GapRows{GSt.hl, GSt.hr};
  } else {
    const int64_t *gl = D.GL + (int64_t)(active ? i : 0) * SD_GAPW * SD_SLOTS;
    const int64_t *gr = D.GR + (int64_t)(active ? j : 0) * SD_GAPW * SD_SLOTS;
    GS = GapRows{reinterpret_cast<const int64_t(*)[SD_SLOTS]>(gl),
                 reinterpret_cast<const int64_t(*)[SD_SLOTS]>(gr)};
  }

  int64_t Bs[SD_SLOTS], PSs[SD_SLOTS];
#pragma unroll
  for (int s = 0; s < SD_SLOTS; s++) {
    Bs[s] = SD_INF;
    PSs[s] = SD_INF;
  }
  // the state pairs of this layer pair, and the most any group of the warp
  // has: the slot loops run that many rounds (warp-uniform: the groups'
  // shuffles need every lane), each group idling past its own count
  const int nslot = active ? wa * wb : 0;
  const int kslot = (int)__reduce_max_sync(FULL, (unsigned)nslot);
#pragma unroll 1
  for (int k = 0; k < kslot; k++) {
    const bool ok = k < nslot;
    const int sa = ok ? k / wb : 0, sb = ok ? k % wb : 0, s = sa * SD_W + sb;
    const int a = a0 + sa, b = b0 + sb;
    const int cell = ok ? F.cs(i, sa, j, sb) : 0;  // this state pair's full-table entry
    // gap cell: thread k of the group takes in-edge k of b
    {
      int64_t hv = SD_INF;
      if (ok) {
        const int nib = F.nin(b);
#pragma unroll 1
        for (int k = sub; k < nib; k += G) {
          const SdEdge e = F.in(b, k);
          const int64_t hp = g == 1 ? (e.other == a ? 0 : SD_INF) : ro(F.H + F.cs(i, sa, j - 1, e.other - js));
          if (!fin(hp)) continue;
          upd(hv, hp + e.cost);
          TERM(1);
        }
      }
      seg_min<G>(hv);
      if (ok && sub == 0) {
        hv = settle(hv);
        D.H[cell] = hv;
        if (g < SD_GAPW) {
          D.GL[((int64_t)i * SD_GAPW + g) * SD_SLOTS + sb * SD_W + sa] = hv;
          D.GR[((int64_t)j * SD_GAPW + g) * SD_SLOTS + sa * SD_W + sb] = hv;
        }
      }
    }
    // Ihat: inner pair (c,d) one nucleotide inside (a,b) and its loop-side mismatch
    {
      int64_t iv = SD_INF;
      if (ok && g >= 7) {
        const int no = F.nout(a), ni = F.nin(b);
#pragma unroll 1
        for (int q = sub; q < no * ni; q += G) {
          const int k2 = q % ni, k1 = q / ni;
          const SdEdge e1 = F.out(a, k1), e2 = F.in(b, k2);
          int64_t vi[6];
          F.v6(F.cs(i + 1, e1.other - i1s, j - 1, e2.other - js), vi);
          const int64_t w = best_inner(vi, T.mmI, e2.label * 4 + e1.label);
          if (!fin(w)) continue;
          upd(iv, w + e1.cost + e2.cost);
          TERM(3);
        }
      }
      seg_min<G>(iv);
      if (ok && sub == 0) D.Ihat[rcell + s] = settle(iv);
    }
    // typed closed values V_t, thread t of the group taking type t (G >= 8),
    // then Eq. (branch) B and the bulge term WB (inner pair (a, b)) as group
    // minima over the types
    {
      const int t = sub;
      int64_t v = SD_INF;
      if (ok && t < 6 && g >= 5) {
        // the pair's 5' and 3' nucleotides; the out-edge of a labelled with the
        // 5' one (a DFA has at most one; out-edges are stored by label)
        const int l5 = (0x323210 >> (4 * t)) & 15, l3 = (0x230123 >> (4 * t)) & 15;
        const int oma = D.out_mask[a];
        if (((oma >> l5) & 1) && ((D.in_mask[b] >> l3) & 1)) {
          const SdEdge e1 = F.out(a, __popc(oma & ((1 << l5) - 1)));
          const int nib = F.nin(b);
#pragma unroll 1
          for (int k2 = 0; k2 < nib; k2++) {
            const SdEdge e2 = F.in(b, k2);
            if (e2.label != l3) continue;
            const int64_t qv = ro(D.Q + F.rs(i + 1, e1.other - i1s, j - 1, e2.other - js) * 6 + t);
            if (!fin(qv)) continue;
            upd(v, qv + e1.cost + e2.cost);
            TERM(2);
          }
        }
      }
      v = settle(v);
      if (ok && t < 6) D.V[(int64_t)cell * 6 + t] = v;
      int64_t B = SD_INF, wbv = SD_INF;
      if (fin(v)) {
        B = v + fx(T.mlintern + T.au[t]);
        wbv = v + fx(T.au[rev_type(t)]);
        TERM(1);
      }
      seg_min<G>(B);
      seg_min<G>(wbv);
      B = settle(B);
      if (ok && sub == 0) {
        D.Bv[cell] = B;
        D.WB[rcell + s] = settle(wbv);
      }
      if (ok) Bs[s] = B;
    }
    // the one-nucleotide-side factors X(a, b) (inner pair (a, d), d -> b) and
    // Y(a, b) (inner pair (c, b), a -> c) of the 1 x n and n x 1 loops
    if (ok) {
      const int im = D.in_mask[a], om = D.out_mask[b];
      const int nib = F.nin(b), noa = F.nout(a);
      const int sp = g & (SD_XSPAN - 1);
      for (int q = sub; q < 8; q += G) {
        const int lab = q & 3;
        int64_t x = SD_INF;
        if (q < 4) {  // X(a, b)[p = lab]: inner pair (a, d) of span g-1
          if (!((im >> lab) & 1)) continue;
          if (g >= 6)
#pragma unroll 1
            for (int k = 0; k < nib; k++) {
              const SdEdge e = F.in(b, k);
              int64_t vi[6];
              F.v6(F.cs(i, sa, j - 1, e.other - js), vi);
              const int64_t t = best_inner(vi, T.mm1n, e.label * 4 + lab);
              if (fin(t)) {
                upd(x, t + e.cost);
                TERM(2);
              }
            }
          D.Xc[((int64_t)(a * 4 + lab) * SD_XSPAN + sp) * SD_W + sb] = settle(x);
        } else {  // Y(a, b)[r = lab]: inner pair (c, b) of span g-1
          if (!((om >> lab) & 1)) continue;
          if (g >= 6)
#pragma unroll 1
            for (int k = 0; k < noa; k++) {
              const SdEdge e = F.out(a, k);
              int64_t vi[6];
              F.v6(F.cs(i + 1, e.other - i1s, j, sb), vi);
              const int64_t t = best_inner(vi, T.mm1n, lab * 4 + e.label);
              if (fin(t)) {
                upd(x, t + e.cost);
                TERM(2);
              }
            }
          D.Yr[((int64_t)(b * 4 + lab) * SD_XSPAN + sp) * SD_W + sa] = settle(x);
        }
      }
    }
    // Two-loop factors Af of this cell (a, b) for the pairs closing one
    // nucleotide outside it (x -> a and b -> y; read by q_slot two spans up).
    // Everything that does not depend on the outer pair is taken once per
    // cell: the inner pair, the unpaired nucleotides beyond a or b and their
    // path costs:
    //   [p]    1 x n: l1 = 1 (nucleotide p enters a), the inner pair (a, d) with
    //          d -> u, u on layer lu, l2 = j + 2 - lu >= 3: X(a,u)[p] + H(u -> b)
    //          + size / asymmetry (by row, after the slot loop)
    //   [4+r]  n x 1: l2 = 1 (nucleotide r leaves b), the inner pair (c, b) with
    //          w -> c, w on layer lw, l1 = lw - i + 2 >= 3: Y(w,b)[r] + H(a -> w)
    //          + size / asymmetry (by column, after the slot loop)
    //   [8]    2 x 3 and 3 x 2: the inner pair's V with its 2x3 mismatch, the
    //          unpaired edges, size (here)
    {
      int64_t af[9];
#pragma unroll
      for (int q = 0; q < 9; q++) af[q] = SD_INF;
      if (ok && g >= 7) {
        if (g >= 8) {
          const int64_t e23 = fx(T.interior[5] + T.ninio);
          // 2 x 3: a -> c (p2) on layer i+1; d on layer j-2 -> u (r1) on j-1; H(u -> b)
          {
            const int noa = F.nout(a);
            const int ro0 = F.fo_off[F.ls(j - 2)], nro = F.fo_off[F.ls(j - 1)] - ro0;
            const int cs0 = F.ls(i + 1), ds0 = F.ls(j - 2), us0 = F.ls(j - 1);
#pragma unroll 1
            for (int k = sub; k < noa * nro; k += G) {
              const int kp = k / nro, kr = k - kp * nro;
              const SdEdge p2 = F.out(a, kp);
              const SdFlatEdge r1 = F.fo[ro0 + kr];
              const int64_t h = GS.hr[1][((r1.wl >> 2) - us0) * SD_W + sb];
              if (!fin(h)) continue;
              int64_t vi[6];
              F.v6(F.cs(i + 1, p2.other - cs0, j - 2, r1.v - ds0), vi);
              const int64_t wv = best_inner(vi, T.mm23, (r1.wl & 3) * 4 + p2.label);
              if (!fin(wv)) continue;
              upd(af[8], wv + p2.cost + r1.cost + h + e23);
              TERM(5);
            }
          }
          // 3 x 2: a -> w (H) on layer i+1, w -> c (p2) on i+2; d on j-1 -> b (r1)
          {
            const int nib = F.nin(b);
            const int po0 = F.fo_off[F.ls(i + 1)], npo = F.fo_off[F.ls(i + 2)] - po0;
            const int ws0 = F.ls(i + 1), cs0 = F.ls(i + 2), ds0 = F.ls(j - 1);
#pragma unroll 1
            for (int k = sub; k < npo * nib; k += G) {
              const int kp = k / nib, kr = k - kp * nib;
              const SdFlatEdge p2 = F.fo[po0 + kp];
              const SdEdge r1 = F.in(b, kr);
              const int64_t h = GS.hl[1][(p2.v - ws0) * SD_W + sa];
              if (!fin(h)) continue;
              int64_t vi[6];
              F.v6(F.cs(i + 2, (p2.wl >> 2) - cs0, j - 1, r1.other - ds0), vi);
              const int64_t wv = best_inner(vi, T.mm23, r1.label * 4 + (p2.wl & 3));
              if (!fin(wv)) continue;
              upd(af[8], wv + p2.cost + r1.cost + h + e23);
              TERM(5);
            }
          }
        }
      }
      seg_min<G>(af[8]);
      if (ok && sub == 0) D.Af[(int64_t)(rcell + s) * SD_AN + 8] = settle(af[8]);
    }
  }
  // The 1 x n factors Af[p] by row (the state a of slot sa with two slots of
  // layer j at a time: the window of u and the X values are the same for the
  // row) and the n x 1 factors Af[4 + r] by column (the state b of slot sb
  // with two slots of layer i at a time).  Item k of the rows is row k / np of
  // the slot pair k % np (np pairs of slots at the other end), likewise for
  // the columns.  acc[side * 4 + label] holds the two slots of the pair; the
  // group minimum leaves value (sub & 7) in thread sub.
  {
    const int npj = SD_W == 2 ? 1 : (wb + 1) / 2, npi = SD_W == 2 ? 1 : (wa + 1) / 2;
    const int nrow = active ? wa * npj : 0, ncol = active ? wb * npi : 0;
    const int kr = (int)__reduce_max_sync(FULL, (unsigned)max(nrow, ncol));
#pragma unroll 1
    for (int k = 0; k < kr; k++) {
      // row item k: row ra of layer i, slots pb, pb + 1 of layer j (1 x n)
      {
        const bool ok = k < nrow;
        const int ra = ok ? k / npj : 0, pb = ok ? 2 * (k % npj) : 0;
        int64_t acc[8];
#pragma unroll
        for (int q = 0; q < 8; q++) acc[q] = SD_INF;
        const int ulo = max(i + 6, j - (SD_MAXTWO - 3)), uhi = j - 1;
        if (ok && g >= 7 && ulo <= uhi) {
          const int a = a0 + ra, im = D.in_mask[a];
          const int uend = F.ls(uhi + 1);
          // 2 states per thread and round, their loads issued together
#pragma unroll 1
          for (int u = F.ls(ulo) + sub; u < uend; u += 2 * G) {
            int64_t h0[2], h1[2], e[2], x[2][4];
#pragma unroll
            for (int v = 0; v < 2; v++) {
              const int uu = u + v * G;
              const bool in = uu < uend;
              const int pu = in ? __ldg(&D.pos[uu]) : 0;
              const int lu = pu >> SD_CAND_SHIFT, us = pu & ((1 << SD_CAND_SHIFT) - 1), l2 = j + 2 - lu;
              h0[v] = in ? GS.hr[j - lu][us * SD_W + pb] : SD_INF;
              h1[v] = in ? GS.hr[j - lu][us * SD_W + pb + 1] : SD_INF;
              e[v] = in ? fx(T.interior[1 + l2] + min(T.maxninio, T.ninio * (l2 - 1))) : 0;
              const bool any = fin(h0[v]) || fin(h1[v]);
              const int64_t *xc =
                  D.Xc + ((int64_t)a * 4 * SD_XSPAN + ((lu - i) & (SD_XSPAN - 1))) * SD_W + us;
#pragma unroll
              for (int p = 0; p < 4; p++)
                x[v][p] = any && ((im >> p) & 1) ? ro(xc + p * SD_XSPAN * SD_W) : SD_INF;
            }
#pragma unroll
            for (int v = 0; v < 2; v++)
#pragma unroll
              for (int p = 0; p < 4; p++) {
                if (!fin(x[v][p])) continue;
                if (fin(h0[v])) {
                  upd(acc[p], x[v][p] + h0[v] + e[v]);
                  TERM(2);
                }
                if (fin(h1[v])) {
                  upd(acc[4 + p], x[v][p] + h1[v] + e[v]);
                  TERM(2);
                }
              }
          }
        }
        const int64_t v = seg_min8<G>(acc, sub);
        const int sb = pb + ((sub >> 2) & 1);
        if (ok && sub < 8 && sb < wb)
          D.Af[(int64_t)(rcell + ra * SD_W + sb) * SD_AN + (sub & 3)] = settle(v);
      }
      // column item k: column cb of layer j, slots pb, pb + 1 of layer i (n x 1)
      {
        const bool ok = k < ncol;
        const int cb = ok ? k / npi : 0, pb = ok ? 2 * (k % npi) : 0;
        int64_t acc[8];
#pragma unroll
        for (int q = 0; q < 8; q++) acc[q] = SD_INF;
        const int wlo = i + 1, whi = min(i + SD_MAXTWO - 3, j - 6);
        if (ok && g >= 7 && wlo <= whi) {
          const int b = b0 + cb, om = D.out_mask[b];
          const int wend = F.ls(whi + 1);
          // 2 states per thread and round, their loads issued together
#pragma unroll 1
          for (int w = F.ls(wlo) + sub; w < wend; w += 2 * G) {
            int64_t h0[2], h1[2], e[2], y[2][4];
#pragma unroll
            for (int v = 0; v < 2; v++) {
              const int ww = w + v * G;
              const bool in = ww < wend;
              const int pw = in ? __ldg(&D.pos[ww]) : 0;
              const int lw = pw >> SD_CAND_SHIFT, ws = pw & ((1 << SD_CAND_SHIFT) - 1), l1 = lw - i + 2;
              h0[v] = in ? GS.hl[lw - i][ws * SD_W + pb] : SD_INF;
              h1[v] = in ? GS.hl[lw - i][ws * SD_W + pb + 1] : SD_INF;
              e[v] = in ? fx(T.interior[l1 + 1] + min(T.maxninio, T.ninio * (l1 - 1))) : 0;
              const bool any = fin(h0[v]) || fin(h1[v]);
              const int64_t *yr =
                  D.Yr + ((int64_t)b * 4 * SD_XSPAN + ((j - lw) & (SD_XSPAN - 1))) * SD_W + ws;
#pragma unroll
              for (int r = 0; r < 4; r++)
                y[v][r] = any && ((om >> r) & 1) ? ro(yr + r * SD_XSPAN * SD_W) : SD_INF;
            }
#pragma unroll
            for (int v = 0; v < 2; v++)
#pragma unroll
              for (int r = 0; r < 4; r++) {
                if (!fin(y[v][r])) continue;
                if (fin(h0[v])) {
                  upd(acc[r], y[v][r] + h0[v] + e[v]);
                  TERM(2);
                }
                if (fin(h1[v])) {
                  upd(acc[4 + r], y[v][r] + h1[v] + e[v]);
                  TERM(2);
                }
              }
          }
        }
        const int64_t v = seg_min8<G>(acc, sub);
        const int sa = pb + ((sub >> 2) & 1);
        if (ok && sub < 8 && sa < wa)
          D.Af[(int64_t)(rcell + sa * SD_W + cb) * SD_AN + 4 + (sub & 3)] = settle(v);
      }
    }
  }
  // IL: generic internal loops (l1 = l1'+2, l2 = l2'+2 unpaired nucleotides,
  // l1'+l2' = m in [2, 26]) below every state pair of the layer pair, by loop
  // size.  K_m(x, y) is the best such loop inside (x, y) with l1'+l2' = m, its
  // asymmetry term included: growing both unpaired sides by one nucleotide
  // keeps |l1 - l2|, so a loop with both sides >= 1 is a loop of K_{m-2} of a
  // state pair one nucleotide inside plus the two edges; a loop with one side
  // empty is an inner mismatch cell (Ihat) on x's column or y's row plus the
  // staged gap of the other side.  IL = min over m of K_m + the size term.
  // K_0..K_24 are kept (ring of 4 spans) for the pairs two spans up.
  __syncwarp();  // this layer pair's own Ihat (m = 0) was written above
#pragma unroll 1
  for (int k = 0; k < kslot; k++) {
    const bool ok = k < nslot;
    const int sa = ok ? k / wb : 0, sb = ok ? k % wb : 0, s = sa * SD_W + sb;
    int64_t il = SD_INF;
    if (ok && g >= 7) {
      const int x = a0 + sa, y = b0 + sb;
      int64_t *Kc = D.KR + ((int64_t)((g & 3) * (n + 1) + i) * SD_SLOTS + s) * SD_KM;
      const int64_t *Kin = D.KR + (int64_t)(((g - 2) & 3) * (n + 1) + i + 1) * SD_SLOTS * SD_KM;
      const int nox = F.nout(x), niy = F.nin(y);
#pragma unroll 1
      for (int m = sub; m <= SD_MAXTWO - 4; m += G) {
        int64_t km = SD_INF;
        const int64_t asym = fx(min(T.maxninio, T.ninio * m));
        // l1' = 0: the inner mismatch cell (x, b), b on layer j - m
        const int lb = j - m;
        if (lb - i >= 7)
          for (int ds = 0; ds < (SD_W == 2 ? SD_W : F.w(lb)); ds++) {
            const int64_t h = GS.hr[m][ds * SD_W + sb];  // +inf past the width
            if (!fin(h)) continue;
            const int r = F.rs(i, sa, lb, ds);
            const int64_t v = m == 0 ? D.Ihat[r] : ro(D.Ihat + r);
            if (fin(v)) {
              upd(km, v + h + asym);
              TERM(2);
            }
          }
        // l2' = 0, l1' = m >= 1: the inner mismatch cell (a, y), a on layer i + m
        const int la = i + m;
        if (m >= 1 && j - la >= 7)
          for (int cs = 0; cs < (SD_W == 2 ? SD_W : F.w(la)); cs++) {
            const int64_t h = GS.hl[m][cs * SD_W + sa];  // +inf past the width
            if (!fin(h)) continue;
            const int64_t v = ro(D.Ihat + F.rs(la, cs, j, sb));
            if (fin(v)) {
              upd(km, v + h + asym);
              TERM(2);
            }
          }
        // both sides >= 1: K_{m-2} of the state pair (x', y') one nucleotide inside
        if (m >= 2 && g >= 9)
#pragma unroll 1
          for (int a2 = 0; a2 < nox; a2++) {
            const SdEdge e1 = F.out(x, a2);
#pragma unroll 1
            for (int b2 = 0; b2 < niy; b2++) {
              const SdEdge e2 = F.in(y, b2);
              const int64_t kv =
                  ro(Kin + ((e1.other - i1s) * SD_W + (e2.other - js)) * SD_KM + m - 2);
              if (fin(kv)) {
                upd(km, kv + e1.cost + e2.cost);
                TERM(2);
              }
            }
          }
        km = settle(km);
        if (m < SD_KM) Kc[m] = km;
        if (m >= 2 && fin(km)) {
          upd(il, km + fx(T.interior[m + 4]));
          TERM(1);
        }
      }
    }
    seg_min<G>(il);
    if (ok && sub == 0) D.IL[rcell + s] = settle(il);
  }
  // Eq. (sparse2) for every slot: edge extensions, then splits at retained
  // candidates (the group splits the candidate list)
#pragma unroll 1
  for (int k = 0; k < kslot; k++) {
    const bool ok = k < nslot;
    const int sa = ok ? k / wb : 0, sb = ok ? k % wb : 0, s = sa * SD_W + sb;
    const int a = a0 + sa, b = b0 + sb;
    const int cell = ok ? F.cs(i, sa, j, sb) : 0;
    int64_t s2 = SD_INF, ps = SD_INF;
    if (ok) {
      // one unpaired edge at either end: the out-edges of a (P_S), then the
      // in-edges of b (P_S and the edge extensions of S2), split over the group
      if (g >= 2) {
        const int noa = F.nout(a), nt = noa + F.nin(b);
#pragma unroll 1
        for (int k = sub; k < nt; k += G) {
          const bool left = k < noa;
          const SdEdge e = left ? F.out(a, k) : F.in(b, k - noa);
          const int c = left ? F.cs(i + 1, e.other - i1s, j, sb) : F.cs(i, sa, j - 1, e.other - js);
          const int64_t v1 = ro(D.S1 + c), v2 = left ? SD_INF : ro(D.S2 + c);
          if (fin(v1)) {
            upd(ps, v1 + e.cost + mlb);
            TERM(2);
          }
          if (fin(v2)) {
            upd(s2, v2 + e.cost + mlb);
            TERM(2);
          }
        }
      }
      const int cnt = D.cand_cap ? min(D.cand_cnt[b], __ldg(&D.cand_cap[b])) : D.cand_cnt[b];
      const int64_t off = D.cand_off[b];
      // two entries per thread and round, their loads issued together (the
      // S1 rows of the splits are far apart: more loads in flight); entries
      // are in decreasing layer order, so the scan ends at the first entry
      // on layer i or before
#pragma unroll 1
      for (int k0 = sub; k0 < cnt; k0 += 2 * G) {
        int ce[2];
        bool in[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
          const int k = k0 + u * G;
          ce[u] = k < cnt ? D.cand_c[off + k] : 0;
          in[u] = k < cnt && (ce[u] >> SD_CAND_SHIFT) > i;
        }
        int64_t v[2], cb[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
          v[u] = in[u] ? ro(D.S1 + F.cs(i, sa, ce[u] >> SD_CAND_SHIFT,
                                        ce[u] & ((1 << SD_CAND_SHIFT) - 1)))
                       : SD_INF;
          cb[u] = in[u] ? D.cand_B[off + k0 + u * G] : 0;
        }
#pragma unroll
        for (int u = 0; u < 2; u++)
          if (fin(v[u])) {
            upd(s2, v[u] + cb[u]);
            TERM(1);
          }
        if (!in[1]) break;
      }
    }
    seg_min<G>(s2);
    s2 = settle(s2);
    // P_S (Eq. partitionable with S): S2 or one unpaired edge at either end
    seg_min<G>(ps);
    if (ok && sub == 0) {
      D.S2[cell] = s2;
      upd(ps, s2);
      ps = settle(ps);
      int64_t s1 = ps;
      if (fin(Bs[s])) upd(s1, Bs[s]);
      D.S1[cell] = s1;
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
            D.cand_c[off + cnt] = (i << SD_CAND_SHIFT) | sa;
            D.cand_B[off + cnt] = Bs[s];
          } else {
            // presized room exceeded: this run is repeated
            atomicOr(reinterpret_cast<unsigned long long *>(&D.tb[3]), (unsigned long long)SD_TB_OVERFLOW);
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
  if constexpr (G == 32 || SD_W > 2) {  // one group per warp (or wide slots): no pooling
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
#pragma unroll
      for (int t = 0; t < 6; t++) qv[t] = SD_INF;
      if (tm) q_slot<G, COUNT>(F, D, P, T, sub, a0 + sa, b0 + sb, i, sa, j, sb, tm, qv, ops, GS);
      const int64_t q8[8] = {qv[0], qv[1], qv[2], qv[3], qv[4], qv[5], SD_INF, SD_INF};
      const int64_t qt = seg_min8<G>(q8, sub);  // type sub & 7
      if (ok && sub < 6) D.Q[(int64_t)(rcell + s) * 6 + sub] = settle(qt);
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
      if (!tm && sub < 6) D.Q[(int64_t)(rcell + s) * 6 + sub] = SD_INF;  // no outer type closes (x, y)
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
#pragma unroll
    for (int t = 0; t < 6; t++) qv[t] = SD_INF;
    const SdDesign &Do = designs[o_dsel];
    const int sa = s_k / SD_W, sb = s_k % SD_W;
    if (tm_k) {
      Fv Fo;
      Fo.n = Do.n;
      Fo.N = Do.N;
      Fo.layout = Do.layout;
      Fo.maxin = Do.maxin;
      Fo.poff = Do.poff;
      Fo.lst = Do.lstart;
      Fo.oe = Do.out;
      Fo.ie = Do.in;
      Fo.on = Do.out_cnt;
      Fo.in_ = Do.in_cnt;
      Fo.H = Do.H;
      Fo.V = Do.V;
      Fo.fo = Do.fo;
      Fo.fo_off = Do.fo_off;
      Fo.fi = Do.fi;
      Fo.fi_off = Do.fi_off;
      const GapStage &og = s_gap[(threadIdx.x >> 5) * NGW + go_k];
      q_slot<G, COUNT>(Fo, Do, P, T, sub, o_a0 + sa, o_b0 + sb, o_i, sa, o_i + g, sb, tm_k, qv,
                       ops, GapRows{og.hl, og.hr});
    }
    const int o_rcell = ((g & (SD_RING - 1)) * (Do.n + 1) + o_i) * SD_SLOTS;
    const int64_t q8[8] = {qv[0], qv[1], qv[2], qv[3], qv[4], qv[5], SD_INF, SD_INF};
    const int64_t qt = seg_min8<G>(q8, sub);  // type sub & 7
    if (tm_k && sub < 6) Do.Q[(int64_t)(o_rcell + s_k) * 6 + sub] = settle(qt);
    if (COUNT && tm_k && ops) atomicAdd(&ops_out[o_dsel], ops);
    ops = 0;
  }
}

// ---------------------------------------------------------------------------
// exterior suffix values (Sec. 5 final-column exterior DP), one block per design
// ---------------------------------------------------------------------------
#ifndef SD_EXT_THREADS
#define SD_EXT_THREADS 1024
#endif
__global__ void __launch_bounds__(SD_EXT_THREADS) k_exterior(const SdDesign *__restrict__ designs,
                                                             const SdParams *__restrict__ Pp) {
  const SdDesign &D = designs[blockIdx.x];
  const SdParams &P = *Pp;
  __shared__ int64_t smv[SD_EXT_THREADS / 32][SD_W];
  Lat G(D);
  const int n = D.n, N = D.N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // a branch (a, b): min over t of V_t + AU(t) = B(a, b) - ML_intern (Eq.
  // branch adds the same ML_intern to every type)
  const int64_t mli = fx(P.mlintern);
  if (threadIdx.x == 0) D.Ext[N - 1] = 0;
  __syncthreads();
  // layer by layer from the end, every state of the layer at once
  for (int k = n - 1; k >= 0; k--) {
    const int a0 = G.lstart(k), wa = G.lstart(k + 1) - a0;
    int64_t bv[SD_W];
#pragma unroll
    for (int s = 0; s < SD_W; s++) bv[s] = SD_INF;
    // unpaired: the out-edges of the layer's states, one per thread
    if ((int)threadIdx.x < wa * SD_MAXOUT) {
      const int sa = threadIdx.x / SD_MAXOUT, q = threadIdx.x % SD_MAXOUT;
      if (q < G.nout(a0 + sa)) {
        const SdEdge e = G.out(a0 + sa, q);
        const int64_t x = D.Ext[e.other];
#pragma unroll
        for (int s = 0; s < SD_W; s++)
          if (s == sa && fin(x)) upd(bv[s], x + e.cost);
      }
    }
    for (int b = G.lstart(min(k + 5, n + 1)) + threadIdx.x; b < N; b += blockDim.x) {
      const int64_t eb = D.Ext[b];
      if (!fin(eb)) continue;
      const int lb = G.layer(b);
#pragma unroll
      for (int s = 0; s < SD_W; s++)
        if (s < wa) {
          const int64_t bb = D.Bv[G.slot(a0 + s, b, k, lb)];
          if (fin(bb)) upd(bv[s], bb - mli + eb);
        }
    }
#pragma unroll
    for (int s = 0; s < SD_W; s++) {
      warp_min(bv[s]);
      if (lane == 0) smv[w][s] = bv[s];
    }
    __syncthreads();
    if ((int)threadIdx.x < wa) {
      int64_t v = SD_INF;
      for (int q = 0; q < (int)(blockDim.x >> 5); q++) upd(v, smv[q][threadIdx.x]);
      D.Ext[a0 + threadIdx.x] = settle(v);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// traceback (Sec. 5), one block per design.  The fill keeps values only, so
// every step re-derives its canonical choice from the full tables: the first
// option, in a fixed enumeration order, whose value equals the cell's value
// (exact integer equality).  The orders:
//   exterior  unpaired out-edge by label, then branch (b ascending, type)
//   V_t(a,b)  for each in-edge of b with the pair's 3' label, in in-edge
//             order: hairpin (special lengths: interior paths in label order;
//             else (first, last) loop labels), two-loops by (l1+l2, l1, c, d,
//             inner type, left side, right side), multiloop
//   B         smallest pair type
//   S2        edge extension (in-edge order), then candidate split at the
//             smallest state c of C_b
//   S1        direct branch, left peel (out-edge order), right peel (in-edge
//             order), two-branch value
//   sides     (first, last) labels; the gap inside by the greedy label order
// Thread 0 walks the structure and owns the work list; the searches over
// many options (exterior branches, two-loops, candidate splits) use the whole
// block and a block-wide minimum of the option's position in the order.
// ---------------------------------------------------------------------------
#ifndef SD_TB_THREADS
#define SD_TB_THREADS 1024
#endif
constexpr int TB_THREADS = SD_TB_THREADS;
constexpr unsigned long long NO_OPTION = ~0ull;

__device__ unsigned long long block_min(unsigned long long v, unsigned long long *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(FULL, v, o);
    v = u < v ? u : v;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < TB_THREADS / 32 ? red[lane] : NO_OPTION;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long u = __shfl_xor_sync(FULL, v, o);
      v = u < v ? u : v;
    }
    if (lane == 0) red[TB_THREADS / 32] = v;
  }
  __syncthreads();
  v = red[TB_THREADS / 32];
  __syncthreads();
  return v;
}

// Unpaired sides of a two-loop: the (first, last) label descriptions of the
// paths x -> y of len edges and their minimum costs.  key: len 0 -> 0; len 1
// -> the label; len >= 2 -> first*4 + last (a DFA has one 2-edge path per
// label pair).  Descriptors come in increasing key order.
struct Sides {
  int cnt;
  uint8_t key[16], first[16], last[16];
  int64_t cost[16];
};

__device__ void side_descs(const Lat &G, int x, int y, int len, Sides &S) {
  S.cnt = 0;
  if (len == 0) {
    if (x == y) {
      S.key[0] = S.first[0] = S.last[0] = 0;
      S.cost[0] = 0;
      S.cnt = 1;
    }
    return;
  }
  if (len == 1) {
    for (int k = 0; k < G.nout(x); k++) {
      const SdEdge e = G.out(x, k);
      if (e.other != y) continue;
      S.key[S.cnt] = S.first[S.cnt] = S.last[S.cnt] = (uint8_t)e.label;
      S.cost[S.cnt++] = e.cost;
    }
    return;
  }
  if (len == 2) {
    for (int k = 0; k < G.nout(x); k++) {
      const SdEdge e = G.out(x, k);
      for (int k2 = 0; k2 < G.nout(e.other); k2++) {
        const SdEdge e2 = G.out(e.other, k2);
        if (e2.other != y) continue;
        S.key[S.cnt] = (uint8_t)(e.label * 4 + e2.label);
        S.first[S.cnt] = (uint8_t)e.label;
        S.last[S.cnt] = (uint8_t)e2.label;
        S.cost[S.cnt++] = e.cost + e2.cost;
      }
    }
    return;
  }
  for (int k = 0; k < G.nout(x); k++) {
    const SdEdge e = G.out(x, k);  // out-edges are stored by label
    for (int l = 0; l < 4; l++) {
      int64_t best = SD_INF;
      for (int q = 0; q < G.nin(y); q++) {
        const SdEdge ei = G.in(y, q);
        if (ei.label != l) continue;
        const int64_t h = G.Hp(e.other, ei.other);
        if (fin(h)) upd(best, e.cost + h + ei.cost);
      }
      if (!fin(best)) continue;
      S.key[S.cnt] = (uint8_t)(e.label * 4 + l);
      S.first[S.cnt] = (uint8_t)e.label;
      S.last[S.cnt] = (uint8_t)l;
      S.cost[S.cnt++] = best;
    }
  }
}

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
    if (pi < 0 || pj >= D.n || D.structure[pi] != '.' || D.structure[pj] != '.') {
      err = 4;
      return;
    }
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
  // realise the unpaired side x -> y of len edges with descriptor key `key`
  // and cost `cost` (as listed by side_descs)
  __device__ void side(int x, int y, int len, int key, int64_t cost) {
    if (len == 0) {
      if (x != y) err = 6;
      return;
    }
    const int f = len == 1 ? key : key >> 2, l = key & 3;
    const int k1 = G.out_with_label(x, f);
    if (k1 < 0) {
      err = 6;
      return;
    }
    const SdEdge e1 = G.out(x, k1);
    if (len == 1) {
      if (e1.other != y || e1.cost != cost) err = 6;
      else emit(x, e1.label, e1.cost);
      return;
    }
    if (len == 2) {
      const int k2 = G.out_with_label(e1.other, l);
      if (k2 < 0 || G.out(e1.other, k2).other != y) {
        err = 6;
        return;
      }
      const SdEdge e2 = G.out(e1.other, k2);
      emit(x, e1.label, e1.cost);
      emit(e1.other, e2.label, e2.cost);
      return;
    }
    for (int q = 0; q < G.nin(y); q++) {
      const SdEdge ei = G.in(y, q);
      if (ei.label != l) continue;
      const int64_t h = G.Hp(e1.other, ei.other);
      if (fin(h) && e1.cost + h + ei.cost == cost) {
        emit(x, e1.label, e1.cost);
        gap(e1.other, ei.other);
        emit(ei.other, ei.label, ei.cost);
        return;
      }
    }
    err = 6;
  }
  // hairpin closed by type t with interior path a1 -> b1 of L edges and value
  // target; realises the first attaining option and returns 1, else 0
  __device__ int hairpin(int a1, int b1, int t, int L, int64_t target) {
    if (L < 3) return 0;
    if (L == 3 || L == 4 || L == 6) {
      // interior paths in label order (depth-first over out-edges by label)
      int st[8], kk[8], ed[8];
      int64_t cst[8];
      uint32_t labs[8];
      int depth = 0;
      st[0] = a1;
      kk[0] = 0;
      cst[0] = 0;
      labs[0] = 0;
      while (depth >= 0) {
        if (depth == L) {
          const int e = hairpin_seq_e(P, D.hp_len, t, labs[L], L);
          if (fx(e) + cst[L] == target) {
            for (int q = 0; q < L; q++) {
              const SdEdge x = G.out(st[q], ed[q]);
              emit(st[q], x.label, x.cost);
            }
            energy += e;
            return 1;
          }
          depth--;
          continue;
        }
        const int v = st[depth];
        const int k = kk[depth]++;
        if (k >= G.nout(v)) {
          depth--;
          continue;
        }
        const SdEdge e = G.out(v, k);
        if (depth + 1 == L ? e.other != b1 : !fin(G.Hp(e.other, b1))) continue;
        ed[depth] = k;
        st[depth + 1] = e.other;
        cst[depth + 1] = cst[depth] + e.cost;
        labs[depth + 1] = (labs[depth] << 2) | (uint32_t)e.label;
        kk[depth + 1] = 0;
        depth++;
      }
      return 0;
    }
    Sides S;
    side_descs(G, a1, b1, L, S);
    for (int q = 0; q < S.cnt; q++) {
      const int e = hairpin_generic_e(P, D.hp_len, t, L, S.first[q], S.last[q]);
      if (fx(e) + S.cost[q] == target) {
        side(a1, b1, L, S.key[q], S.cost[q]);
        energy += e;
        return 1;
      }
    }
    return 0;
  }
};

// (l1+l2, l1) pairs of the two-loops in enumeration order: pair u has
// l = floor((sqrt(8u+1)-1)/2), l1 = u - l(l+1)/2
constexpr int TL_PAIRS = (SD_MAXTWO + 1) * (SD_MAXTWO + 2) / 2;

// Block-wide search for the first two-loop closing pair type t over the
// interior a1 -> b1 with value target.  Returns the option's position in
// the enumeration order, (((u*W + cs)*W + ds)*6 + ti)*256 + left key*16 + right
// key, or NO_OPTION.
__device__ unsigned long long search_twoloop(const Lat &G, const SdParams &P, int a1, int b1, int t,
                                             int64_t target, unsigned long long *red) {
  unsigned long long best = NO_OPTION;
  const int lx = G.layer(a1), ly = G.layer(b1);
  for (int u4 = threadIdx.x; u4 < TL_PAIRS * SD_SLOTS; u4 += TB_THREADS) {
    const int u = u4 / SD_SLOTS, cs = (u4 / SD_W) % SD_W, ds = u4 % SD_W;
    int l = 0;
    while ((l + 1) * (l + 2) / 2 <= u) l++;
    const int l1 = u - l * (l + 1) / 2, l2 = l - l1;
    const int lc = lx + l1, ld = ly - l2;
    if (ld - lc < 5) continue;
    if (cs >= G.lstart(lc + 1) - G.lstart(lc) || ds >= G.lstart(ld + 1) - G.lstart(ld)) continue;
    const int c = G.lstart(lc) + cs, d = G.lstart(ld) + ds;
    const int64_t hl = G.Hp(a1, c), hr = G.Hp(d, b1);
    if (!fin(hl) || !fin(hr)) continue;
    const int64_t cell = G.slot(c, d, lc, ld) * 6;
    int64_t vv[6], vmin = SD_INF;
    for (int ti = 0; ti < 6; ti++) {
      vv[ti] = G.D.V[cell + ti];
      if (fin(vv[ti])) upd(vmin, vv[ti]);
    }
    // no option of this unit can reach the target: every side costs at
    // least the minimum path cost, every loop at least lb2
    const int64_t floor = hl + hr + fx(P.lb2[l1][l2]);
    if (!fin(vmin) || vmin + floor > target) continue;
    Sides SL, SR;
    side_descs(G, a1, c, l1, SL);
    side_descs(G, d, b1, l2, SR);
    bool found = false;
    for (int ti = 0; ti < 6 && !found; ti++) {
      if (!fin(vv[ti]) || vv[ti] + floor > target) continue;
      for (int p = 0; p < SL.cnt && !found; p++)
        for (int r = 0; r < SR.cnt && !found; r++) {
          const int e = sd_twoloop_energy(P, t, ti, l1, l2, SL.first[p], SL.last[p], SR.first[r],
                                          SR.last[r]);
          if (vv[ti] + fx(e) + SL.cost[p] + SR.cost[r] == target) {
            const unsigned long long pos =
                ((((unsigned long long)u4) * 6 + ti) * 256) + SL.key[p] * 16 + SR.key[r];
            best = pos < best ? pos : best;
            found = true;
          }
        }
    }
  }
  return block_min(best, red);
}

__global__ void __launch_bounds__(TB_THREADS) k_traceback(const SdDesign *__restrict__ designs,
                                                          const SdParams *__restrict__ Pp) {
  const SdDesign &D = designs[blockIdx.x];
  const SdParams &P = *Pp;
  __shared__ unsigned long long red[TB_THREADS / 32 + 1];
  __shared__ int cmd[6];
  __shared__ int64_t cval[2];
  for (int k = threadIdx.x; k < D.n; k += blockDim.x) {
    D.mrna[k] = 0;
    D.structure[k] = '.';
  }
  __syncthreads();
  const bool t0 = threadIdx.x == 0;
  Tb tb(D, P);
  Lat &G = tb.G;
  const int N = D.N;
  if (t0) {
    D.mrna[D.n] = 0;
    D.structure[D.n] = 0;
    if (!fin(D.Ext[0])) tb.err = 14;
  }
  // ---- exterior walk from the source ----
  int a = 0;
  for (int it = 0; it <= D.n + 1; it++) {
    if (t0) {
      cmd[0] = 0;  // 0 done, 1 moved, 2 search branches
      if (a != N - 1 && !tb.err) {
        const int64_t v = D.Ext[a];
        cmd[0] = 2;
        for (int k = 0; k < G.nout(a); k++) {
          const SdEdge e = G.out(a, k);
          const int64_t x = D.Ext[e.other];
          if (fin(x) && x + e.cost == v) {
            tb.emit(a, e.label, e.cost);
            a = e.other;
            cmd[0] = 1;
            break;
          }
        }
      }
      cmd[1] = a;
    }
    __syncthreads();
    const int c0 = cmd[0];
    a = cmd[1];
    __syncthreads();
    if (c0 == 0) break;
    if (c0 == 1) continue;
    // branch (b ascending, type) with V_t(a,b) + AU(t) + Ext(b) = Ext(a): the
    // smallest b with B(a,b) - ML_intern + Ext(b) = Ext(a) (B - ML_intern is
    // the minimum over t of V_t + AU(t)), then its smallest attaining type
    unsigned long long best = NO_OPTION;
    const int la = G.layer(a);
    const int64_t v = D.Ext[a], mli = fx(P.mlintern);
    for (int b = G.lstart(min(la + 5, D.n + 1)) + threadIdx.x; b < N; b += TB_THREADS) {
      const int64_t eb = D.Ext[b];
      if (!fin(eb)) continue;
      const int64_t bb = D.Bv[G.slot(a, b, la, G.layer(b))];
      if (fin(bb) && bb - mli + eb == v) {
        best = (unsigned long long)b;
        break;  // this thread's later b are larger
      }
    }
    best = block_min(best, red);
    if (t0) {
      int t = -1;
      if (best != NO_OPTION) {
        const int b = (int)best;
        const int64_t eb = D.Ext[b], cs = G.slot(a, b, la, G.layer(b)) * 6;
        for (int q = 0; q < 6 && t < 0; q++) {
          const int64_t x = D.V[cs + q];
          if (fin(x) && x + fx(P.au[q]) + eb == v) t = q;
        }
      }
      if (t < 0) {
        tb.err = 15;
      } else {
        const int b = (int)best;
        tb.energy += P.au[t];
        tb.push(1, a, b, t);
        a = b;
      }
      cmd[1] = a;
    }
    __syncthreads();
    a = cmd[1];
    __syncthreads();
  }
  // ---- the work list: 1 V_t(x,y), 2 S1(x,y), 3 S2(x,y), 4 B(x,y) ----
  const int bound = 8 * D.n + 64;
  for (int it = 0; it < bound; it++) {
    if (t0) {
      cmd[0] = 0;
      if (!tb.err && tb.sp > 0) {
        const int32_t *s = D.tb_stack + 4 * --tb.sp;
        cmd[0] = s[0];
        cmd[1] = s[1];
        cmd[2] = s[2];
        cmd[3] = s[3];
      }
      if (it == bound - 1 && cmd[0]) tb.err = 17;
    }
    __syncthreads();
    const int type = cmd[0], x = cmd[1], y = cmd[2], t = cmd[3];
    __syncthreads();
    if (type == 0) break;
    if (type == 4) {  // B(x,y): smallest pair type
      if (t0) {
        const int64_t s = G.slot(x, y, G.layer(x), G.layer(y));
        int tt = 0;
        for (; tt < 6; tt++) {
          const int64_t vv = G.Vt(x, y, tt);
          if (fin(vv) && vv + fx(P.mlintern + P.au[tt]) == D.Bv[s]) break;
        }
        if (tt == 6) {
          tb.err = 9;
        } else {
          tb.energy += P.mlintern + P.au[tt];
          tb.push(1, x, y, tt);
        }
      }
      continue;
    }
    if (type == 2) {  // S1(x,y): direct < left peel < right peel < S2
      if (t0) {
        const int64_t mlb = fx(P.mlbase);
        int xa = x, yb = y, steps = 0;
        while (!tb.err) {
          if (++steps > 2 * D.n + 4) {
            tb.err = 12;
            break;
          }
          const int la = G.layer(xa), lb = G.layer(yb);
          if (lb <= la) {
            tb.err = 12;
            break;
          }
          const int64_t s = G.slot(xa, yb, la, lb);
          const int64_t v = D.S1[s];
          if (!fin(v)) {
            tb.err = 12;
            break;
          }
          if (D.Bv[s] == v) {
            tb.push(4, xa, yb, 0);
            break;
          }
          int moved = 0;
          for (int k = 0; k < G.nout(xa) && !moved; k++) {
            const SdEdge e = G.out(xa, k);
            const int64_t w = G.S1(e.other, yb);
            if (fin(w) && w + e.cost + mlb == v) {
              tb.emit(xa, e.label, e.cost);
              tb.energy += P.mlbase;
              xa = e.other;
              moved = 1;
            }
          }
          for (int k = 0; k < G.nin(yb) && !moved; k++) {
            const SdEdge e = G.in(yb, k);
            const int64_t w = G.S1(xa, e.other);
            if (fin(w) && w + e.cost + mlb == v) {
              tb.emit(e.other, e.label, e.cost);
              tb.energy += P.mlbase;
              yb = e.other;
              moved = 1;
            }
          }
          if (moved) continue;
          if (D.S2[s] == v) tb.push(3, xa, yb, 0);
          else tb.err = 13;
          break;
        }
      }
      continue;
    }
    if (type == 3) {  // S2(x,y): edge extensions, then the candidate split
      if (t0) {
        const int64_t mlb = fx(P.mlbase);
        int yb = y, steps = 0;
        cmd[4] = -1;
        while (!tb.err) {
          if (++steps > D.n + 2) {
            tb.err = 10;
            break;
          }
          const int la = G.layer(x), lb = G.layer(yb);
          const int64_t v = lb > la ? D.S2[G.slot(x, yb, la, lb)] : SD_INF;
          if (!fin(v)) {
            tb.err = 10;
            break;
          }
          int moved = 0;
          for (int k = 0; k < G.nin(yb); k++) {
            const SdEdge e = G.in(yb, k);
            const int64_t w = G.S2(x, e.other);
            if (fin(w) && w + e.cost + mlb == v) {
              tb.emit(e.other, e.label, e.cost);
              tb.energy += P.mlbase;
              yb = e.other;
              moved = 1;
              break;
            }
          }
          if (moved) continue;
          cmd[4] = yb;
          cval[0] = v;
          break;
        }
      }
      __syncthreads();
      const int yb = cmd[4];
      const int64_t v = cval[0];
      __syncthreads();
      if (yb < 0) continue;
      // smallest candidate c of C_yb with S1(x,c) + B(c,yb) = S2(x,yb)
      unsigned long long best = NO_OPTION;
      const int lx = G.layer(x);
      const int cnt = D.cand_cap ? min(D.cand_cnt[yb], D.cand_cap[yb]) : D.cand_cnt[yb];
      const int64_t off = D.cand_off[yb];
      for (int k = threadIdx.x; k < cnt; k += TB_THREADS) {
        const int ce = D.cand_c[off + k], lc = ce >> SD_CAND_SHIFT;
        if (lc <= lx) continue;
        const int c = G.lstart(lc) + (ce & ((1 << SD_CAND_SHIFT) - 1));
        const int64_t w = G.S1(x, c);
        if (fin(w) && w + D.cand_B[off + k] == v) best = (unsigned long long)c < best ? c : best;
      }
      best = block_min(best, red);
      if (t0) {
        if (best == NO_OPTION) {
          tb.err = 11;
        } else {
          tb.push(2, x, (int)best, 0);
          tb.push(4, (int)best, yb, 0);
        }
      }
      continue;
    }
    // type 1: V_t(x,y)
    {
      const int64_t s = G.slot(x, y, G.layer(x), G.layer(y));
      const int64_t v = D.V[s * 6 + t];
      const int kx = G.out_with_label(x, c_pair5[t]);
      if (!fin(v) || kx < 0 || G.layer(y) - G.layer(x) < 5) {
        if (t0) tb.err = 7;
        continue;
      }
      const SdEdge ex = G.out(x, kx);
      const int a1 = ex.other;
      int done = 0;
      for (int k = 0; k < G.nin(y) && !done; k++) {
        const SdEdge ey = G.in(y, k);
        if (ey.label != c_pair3[t]) continue;
        const int b1 = ey.other;
        const int L = G.layer(b1) - G.layer(a1);
        const int64_t target = v - ex.cost - ey.cost;
        if (t0) cmd[5] = tb.hairpin(a1, b1, t, L, target);
        __syncthreads();
        done = cmd[5];
        __syncthreads();
        if (!done) {
          const unsigned long long pos = search_twoloop(G, P, a1, b1, t, target, red);
          if (pos != NO_OPTION) {
            done = 1;
            if (t0) {
              const int rk = (int)(pos & 15), lk = (int)((pos >> 4) & 15);
              const int ti = (int)((pos >> 8) % 6);
              const int u4 = (int)((pos >> 8) / 6), u = u4 / SD_SLOTS;
              const int cs = (u4 / SD_W) % SD_W, ds = u4 % SD_W;
              int l = 0;
              while ((l + 1) * (l + 2) / 2 <= u) l++;
              const int l1 = u - l * (l + 1) / 2, l2 = l - l1;
              const int lc = G.layer(a1) + l1, ld = G.layer(b1) - l2;
              const int c = G.lstart(lc) + cs, d = G.lstart(ld) + ds;
              Sides SL, SR;
              side_descs(G, a1, c, l1, SL);
              side_descs(G, d, b1, l2, SR);
              int p = 0, r = 0;
              while (p < SL.cnt && SL.key[p] != lk) p++;
              while (r < SR.cnt && SR.key[r] != rk) r++;
              if (p == SL.cnt || r == SR.cnt) {
                tb.err = 8;
              } else {
                tb.side(a1, c, l1, lk, SL.cost[p]);
                tb.side(d, b1, l2, rk, SR.cost[r]);
                tb.energy += sd_twoloop_energy(P, t, ti, l1, l2, SL.first[p], SL.last[p],
                                               SR.first[r], SR.last[r]);
                tb.push(1, c, d, ti);
              }
            }
          }
        }
        if (!done && L >= 1) {
          const int64_t s2 = G.S2(a1, b1);
          if (fin(s2) && s2 + fx(P.mlclosing + P.mlintern + P.au[t]) == target) {
            done = 1;
            if (t0) {
              tb.energy += P.mlclosing + P.mlintern + P.au[t];
              tb.push(3, a1, b1, 0);
            }
          }
        }
        if (done && t0) {
          tb.set_pair(G.layer(x), G.layer(y) - 1);
          tb.emit(x, ex.label, ex.cost);
          tb.emit(b1, ey.label, ey.cost);
        }
      }
      if (!done && t0) tb.err = 8;
    }
  }
  if (t0) {
    if (!tb.err && tb.sp > 0) tb.err = 17;
    for (int k = 0; k < D.n && !tb.err; k++)
      if (D.mrna[k] == 0) tb.err = 16;
    D.tb[0] = tb.energy;
    D.tb[1] = tb.pathcost;
    D.tb[2] = tb.err;
  }
}

// Start of a run: empty candidate lists, overflow flag clear, the position of
// every state, gap mirrors reset to the identity (span 0) and +inf.
__global__ void k_clear(const SdDesign *__restrict__ designs) {
  const SdDesign &D = designs[blockIdx.y];
  const int stride = gridDim.x * blockDim.x, t0 = blockIdx.x * blockDim.x + threadIdx.x;
  for (int v = t0; v < D.N; v += stride) {
    D.cand_cnt[v] = 0;
    const int l = D.layer[v];
    D.pos[v] = (l << SD_CAND_SHIFT) | (v - D.lstart[l]);
  }
  if (t0 == 0) D.tb[3] = 0;
  const int64_t total = (int64_t)(D.n + 1) * SD_GAPW * SD_SLOTS;
  for (int64_t e = t0; e < total; e += stride) {
    const int q = (int)(e % SD_SLOTS), l = (int)((e / SD_SLOTS) % SD_GAPW);
    const int x = (int)(e / ((int64_t)SD_SLOTS * SD_GAPW));
    const int c = q / SD_W, sn = q % SD_W;
    const int64_t v = l == 0 && c == sn && sn < D.lstart[x + 1] - D.lstart[x] ? 0 : SD_INF;
    D.GL[e] = v;
    D.GR[e] = v;
  }
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
      const int span = lb - (D.cand_c[off + q] >> SD_CAND_SHIFT);
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
      const int a0 = G.lstart(i), b0 = G.lstart(j);
      for (int sa = 0; sa < wa; sa++)
        for (int sb = 0; sb < wb; sb++) {
          const int64_t s = G.slot(a0 + sa, b0 + sb, i, j);
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
void launch_span(int g, int nact, int64_t items, const SdDesign *d_designs, const int32_t *d_cpre,
                 const SdParams *d_params, cudaStream_t st, unsigned long long *d_ops) {
  constexpr int per_block = FillShape<G>::pairs;
  dim3 grid((unsigned)((items + per_block - 1) / per_block));
  k_fill_span<G, COUNT><<<grid, FillShape<G>::threads, 0, st>>>(d_designs, d_params, g, nact,
                                                                (int)items, d_cpre, d_ops);
}

// Spans g = 1 .. the longest design (designs sorted by length, longest
// first); a design shorter than g drops out.  f(g, nact, items) launches one.
template <class Fn>
void for_each_span(int count, const int *ns, Fn f) {
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
    f(g, nact, items);
  }
}

// Group SD_GROUP_BY_SPAN: 8 threads per layer pair while a span fills the GPU
// with resident group-8 blocks, then 16 while it fills it with group-16
// blocks, then 32: the late spans, too small for one wave, give each layer
// pair more threads (shorter dependent-load chains).
template <bool COUNT>
int span_waves(int64_t &wave8, int64_t &wave16) {
  int dev = 0, sms = 0, b8 = 0, b16 = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b8, k_fill_span<8, COUNT>,
                                                    FillShape<8>::threads, 0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b16, k_fill_span<16, COUNT>,
                                                    FillShape<16>::threads, 0) != cudaSuccess)
    return -1;
  wave8 = (int64_t)sms * b8 * FillShape<8>::pairs;
  wave16 = (int64_t)sms * b16 * FillShape<16>::pairs;
  return 0;
}

template <bool COUNT>
int launch_fill(int G, const SdDesign *d_designs, int count, const int *ns, const int32_t *d_cpre,
                const SdParams *d_params, cudaStream_t st, unsigned long long *d_ops) {
  if (SD_W > 2) G = 32;  // the wide instance has one group size
#if SD_W == 2
  if (G == SD_GROUP_BY_SPAN) {
    int64_t wave8 = 0, wave16 = 0;
    if (span_waves<COUNT>(wave8, wave16)) return -1;
    for_each_span(count, ns, [&](int g, int nact, int64_t items) {
      if (items >= wave8)
        launch_span<8, COUNT>(g, nact, items, d_designs, d_cpre, d_params, st, d_ops);
      else if (items >= wave16)
        launch_span<16, COUNT>(g, nact, items, d_designs, d_cpre, d_params, st, d_ops);
      else
        launch_span<32, COUNT>(g, nact, items, d_designs, d_cpre, d_params, st, d_ops);
    });
    return 0;
  }
#endif
  if (!(G == 32 || (SD_W == 2 && (G == 8 || G == 16)))) return -1;
  for_each_span(count, ns, [&](int g, int nact, int64_t items) {
#if SD_W == 2
    if (G == 8) launch_span<8, COUNT>(g, nact, items, d_designs, d_cpre, d_params, st, d_ops);
    else if (G == 16) launch_span<16, COUNT>(g, nact, items, d_designs, d_cpre, d_params, st, d_ops);
    else
#endif
      launch_span<32, COUNT>(g, nact, items, d_designs, d_cpre, d_params, st, d_ops);
  });
  return 0;
}

}  // namespace

extern "C" int SD_KFN(sd_k_retention)(const SdDesign *d_designs, int item, int32_t *d_hist, int ncodons,
                              void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_hist, 0, sizeof(int32_t) * 8 * (ncodons > 0 ? ncodons : 1), st) !=
      cudaSuccess)
    return -1;
  k_retention<<<64, 256, 0, st>>>(d_designs, item, d_hist);
  if (cudaGetLastError() != cudaSuccess) return -1;
  return cudaStreamSynchronize(st) == cudaSuccess ? 0 : -1;
}

extern "C" int SD_KFN(sd_k_count)(const SdDesign *d_designs, int count, int64_t *d_out, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_out, 0, sizeof(int64_t) * 4 * count, st) != cudaSuccess) return -1;
  k_count<<<dim3(64, count), 256, 0, st>>>(d_designs, (unsigned long long *)d_out);
  if (cudaGetLastError() != cudaSuccess) return -1;
  return cudaStreamSynchronize(st) == cudaSuccess ? 0 : -1;
}

// Counting pass: the same fill with algorithmic-work counters (INT32 slots
// per design, see TERM); the result tables are identical to sd_k_run's.
extern "C" int SD_KFN(sd_k_count_ops)(const SdDesign *d_designs, int count, const int *ns,
                              const int32_t *d_cpre, const SdParams *d_params,
                              unsigned long long *d_ops, void *stream, int group) {
  cudaStream_t st = (cudaStream_t)stream;
  if (count <= 0) return 0;
  if (cudaMemsetAsync(d_ops, 0, sizeof(unsigned long long) * count, st) != cudaSuccess) return -1;
  k_clear<<<dim3(64, count), 256, 0, st>>>(d_designs);
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

extern "C" int SD_KFN(sd_k_run)(const SdDesign *d_designs, int count, const int *ns, const int32_t *d_cpre,
                        const SdParams *d_params, void *stream, int64_t *launches,
                        void *const *events, int group) {
  cudaStream_t st = (cudaStream_t)stream;
  if (count <= 0) {
    if (launches) *launches = 0;
    return 0;
  }
  k_clear<<<dim3(64, count), 256, 0, st>>>(d_designs);
  if (events) record(events[0], st);
  if (launch_fill<false>(group, d_designs, count, ns, d_cpre, d_params, st, nullptr)) return -1;
  if (events) record(events[1], st);
  k_exterior<<<count, SD_EXT_THREADS, 0, st>>>(d_designs, d_params);
  if (events) record(events[2], st);
  k_traceback<<<count, TB_THREADS, 0, st>>>(d_designs, d_params);
  if (events) record(events[3], st);
  if (launches) *launches = (int64_t)ns[0] + 3;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
