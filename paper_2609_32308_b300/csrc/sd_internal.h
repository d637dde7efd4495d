// sd_internal.h -- data layout shared by the host library and the kernels.
//
// Lattice: the layered codon DFA of Sec. 3.  States are numbered layer by
// layer; lstart[l] is the first state of layer l (lstart[n+1] = N).  Every
// layer holds at most SD_W states (the codon trie of the standard code has
// width 2: Leu, Ser, Arg and the stop have two first nucleotides / prefixes).
//
// Tables are "forward packed" by span (the paper's packed layout omits the
// reverse-layer slots): the cells of layer pair (i, i+g), g >= 1, form
// diagonal g; diagonal g starts at cell D(g) = (g-1)(n+1) - (g-1)g/2 and
// layer pair (i, i+g) is cell D(g) + i.  Each cell holds SD_W * SD_W state-pair
// slots (slot = sa*SD_W + sb, sa/sb = state offsets inside their layers), so a
// warp working on consecutive i of one diagonal touches consecutive memory.
#pragma once
#include <stdint.h>

// Layer width of the kernels' layout: the codon trie has width 2; the
// library also builds the kernels for width 8 (sd_kernels_wide.cu) for the
// product of the codon DFA with a forbidden-motif automaton.
#ifndef SD_W
#define SD_W 2
#endif
#define SD_W_WIDE 8
#define SD_SLOTS (SD_W * SD_W)
#define SD_MAXOUT 4      // out-edges per state (one per label in a DFA)
#define SD_MAXIN 8       // in-edges per state of a codon trie (at most 6)
#define SD_MAXIN_WIDE 32 // in-edges per state of a product lattice
#define SD_RING 32       // diagonals kept for the windowed two-loop tables
#define SD_MAXTWO 30     // max unpaired nucleotides in a bulge / internal loop
#ifndef SD_GROUP_BY_SPAN
#define SD_GROUP_BY_SPAN 0  // fill group chosen per span by its layer pairs (as in sd.h)
#endif
#define SD_CAND_SHIFT 3  // slot bits of a candidate entry (layers hold at most 8 states)
#define SD_GAPW (SD_MAXTWO + 1)  // spans 0..SD_MAXTWO of the gap mirrors GL / GR
#define SD_AN 12         // two-loop factor entries per cell slot (9 used, 96 bytes)
#define SD_XSPAN 32      // spans kept per state in the 1 x n / n x 1 factor tables
#define SD_KM 25         // internal-loop sizes kept per state pair for extension
#define SD_KRING 4       // spans kept of them
#define SD_MAX_NT 12000  // longest mRNA: keeps every table index inside int32

// +infinity and the finiteness threshold of the fixed-point arithmetic.
// Stored values are either SD_INF or finite with |v| < 2^57 (checked on the
// host before a design runs), so a sum of at most four stored operands is
// finite iff it is < 2^59, and never overflows.
#define SD_INF (1LL << 60)
#define SD_FINLIM (1LL << 59)
// flags in tb[3] of a design (set by the fill, cleared at the start of a run)
#define SD_TB_OVERFLOW 1  // a presized candidate list overflowed: the run is repeated
#define SD_TB_WAIT 2      // a bounded wait of the fill gave up: the run is invalid
#define SD_EXT_INF (1LL << 62)   // +inf in the dense dump layout

struct SdEdge {
  int32_t other;   // target state (out-edges) or source state (in-edges)
  int32_t label;   // nucleotide 0..3 = A C G U
  int64_t cost;    // fixed-point codon cost (non-zero only on 3rd codon edges)
};

// An edge in a flat list: the out-edges of all states by (source, label), or
// the in-edges by (target, label, source).  States are numbered layer by
// layer, so the edges leaving (entering) the states of layers l0..l1 form one
// contiguous range of the list.
struct SdFlatEdge {
  int32_t v;       // the state whose list holds the edge (source, resp. target)
  int32_t wl;      // the other end * 4 + label
  int64_t cost;
};

// Nearest-neighbour parameters on the device (integer dcal/mol).
struct SdParams {
  int32_t stack[6][6];
  int32_t mmH[6][16], mmI[6][16], mm1n[6][16], mm23[6][16];
  int32_t int11[6][6][16];
  int32_t int21[6][6][64];
  int32_t int22[6][6][256];
  int32_t bulge[32], interior[32];
  int32_t au[6];
  int32_t ninio, maxninio, mlclosing, mlintern, mlbase;
  int32_t nspecial[3];          // triloops (5 nt), tetraloops (6 nt), hexaloops (8 nt)
  int32_t special_code[3][64];  // 2 bits per nucleotide, first nucleotide lowest
  int32_t special_e[3][64];
  // lower bound of the two-loop energy over pair types and loop nucleotides,
  // per (l1, l2) with l1 + l2 <= 30 (prunes the traceback's option search)
  int32_t lb2[SD_MAXTWO + 1][SD_MAXTWO + 1];
};

#ifdef __CUDACC__
#define SD_HD __host__ __device__
#else
#define SD_HD
#endif

// Oriented pair types AU CG GC UA GU UG: 5' / 3' nucleotides and the type of
// the same pair read from the other side.
SD_HD inline int sd_pair5(int t) { return t < 4 ? t : t - 2; }
SD_HD inline int sd_pair3(int t) { return t < 4 ? 3 - t : 7 - t; }
SD_HD inline int sd_rev(int t) { return t < 4 ? 3 - t : 9 - t; }

// Two-loop energy of the Sec. 3 model (dangle-0 reading): t outer pair, ti
// inner pair (5'->3' in the sequence), l1 / l2 unpaired on the 5' / 3' side,
// xi1 = nucleotide after the outer 5' end, xp1 = before the inner 5' end,
// xq1 = after the inner 3' end, xj1 = before the outer 3' end (only those that
// exist are read).
SD_HD inline int sd_twoloop_energy(const SdParams &P, int t, int ti, int l1, int l2, int xi1,
                                   int xp1, int xq1, int xj1) {
  const int s = sd_rev(ti);
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
  const int asym = P.ninio * d < P.maxninio ? P.ninio * d : P.maxninio;
  if (l1 == 1 || l2 == 1)
    return P.interior[l1 + l2] + asym + P.mm1n[t][xi1 * 4 + xj1] + P.mm1n[s][xq1 * 4 + xp1];
  if ((l1 == 2 && l2 == 3) || (l1 == 3 && l2 == 2))
    return P.interior[5] + P.ninio + P.mm23[t][xi1 * 4 + xj1] + P.mm23[s][xq1 * 4 + xp1];
  return P.interior[l1 + l2] + asym + P.mmI[t][xi1 * 4 + xj1] + P.mmI[s][xq1 * 4 + xp1];
}

// One design resident on the device.
struct SdDesign {
  int32_t n, N;           // nucleotides, states
  int32_t status_slot;    // index into the plan's status array
  int32_t dense;          // 1: retain every finite direct interval (scalar-dense control)
  const int32_t *lstart;  // n+2
  const int32_t *layer;   // N
  int32_t *pos;           // N: (layer << SD_CAND_SHIFT) | slot on the layer (set by k_clear)
  const SdEdge *out;      // N * SD_MAXOUT, by label
  const uint8_t *out_cnt; // N
  const SdEdge *in;       // N * maxin, by (label, source)
  const uint8_t *in_cnt;  // N
  const uint8_t *in_mask; // N, bit l set iff some edge with label l enters the state
  const uint8_t *out_mask;// N, bit l set iff the state has an out-edge with label l
  const int32_t *hp_len;  // hairpin length energy for L = 0..n (lxc extrapolation > 30)
  const SdFlatEdge *fo;   // E out-edges by (source, label)
  const int32_t *fo_off;  // N+1: out-edges of state v are fo[fo_off[v] .. fo_off[v+1])
  const SdFlatEdge *fi;   // E in-edges by (target, label, source)
  const int32_t *fi_off;  // N+1
  // Values only: the traceback re-derives every canonical choice from the
  // full tables H, V, B, S1, S2 and the candidate lists.
  int64_t *H;             // ncell*SLOTS  min path cost between states
  int64_t *V;             // ncell*SLOTS*6 typed closed values V_t(a,b)
  int64_t *S1, *S2;       // ncell*SLOTS  sparse one- / two-branch multiloop values
  int64_t *Bv;            // ncell*SLOTS  branch interface B(a,b) = min_t V_t + beta_t
  int64_t *Ihat;          // SD_RING*(n+1)*SLOTS inner pair + its loop-side mismatch
  int64_t *IL;            // SD_RING*(n+1)*SLOTS generic internal loops below a pair
  int64_t *Q;             // SD_RING*(n+1)*SLOTS*6 closed-interior values per outer type
  // SD_RING*(n+1)*SLOTS bulge inner term of each cell (c,d): the minimum over
  // the inner pair types of V plus the terminal penalty of the inner pair
  int64_t *WB;
  // One-nucleotide-side factors of the 1 x n and n x 1 loops, stored by
  // state so that a window of 32 consecutive spans is contiguous (ring by span):
  //   Xc[((a*4 + p)*32 + span)*W + slot of u]: for the cell (a, u), the minimum
  //     over the in-edges d -> u (label fR) of the edge cost plus the minimum
  //     over inner types of V(a,d) + mismatch1n(label fR after d, p before a)
  //   Yr[((b*4 + r)*32 + span)*W + slot of w]: for the cell (w, b), the minimum
  //     over the out-edges w -> c (label lL) of the edge cost plus the minimum
  //     over inner types of V(c,b) + mismatch1n(r after b, lL before c)
  // (N*4*32*W each, W the layer width of the kernel instance)
  int64_t *Xc, *Yr;
  // SD_KRING*(n+1)*SLOTS*SD_KM best generic internal loops of each state pair
  // by size m = l1'+l2' (0..24), asymmetry included (grown two spans up)
  int64_t *KR;
  // SD_RING*(n+1)*SLOTS*SD_AN two-loop factors of each cell (a, b) for the
  // pairs closing one nucleotide outside it (read two spans up): [p] the
  // 1 x n loops (one unpaired nucleotide p entering a, >= 3 after b's side),
  // [4 + r] the n x 1 loops (r leaving b), [8] the 2 x 3 and 3 x 2 loops;
  // each without the outer pair's own mismatch and edge costs
  int64_t *Af;
  // Gap values near the diagonal by layer, (n+1)*SD_GAPW*SLOTS each, so that
  // the fill stages the gap vectors of both ends of a layer pair with
  // contiguous loads: GL[(x*SD_GAPW + l)*SLOTS + c*W + s] = H(slot s of layer
  // x -> slot c of layer x+l), GR[(y*SD_GAPW + l)*SLOTS + c*W + s] = H(slot c
  // of layer y-l -> slot s of layer y); l = 0 holds the identity (0 on the
  // diagonal), empty slots +inf.  Reset at the start of every run, entries of
  // span l written by the fill of span l.
  int64_t *GL, *GR;
  int32_t *cand_cnt;      // N   |C_b|
  const int64_t *cand_off;// N   first entry of C_b
  const int32_t *cand_cap;// N   entries reserved for C_b, or null when each list has its
                          //     worst-case room; a list that outgrows a presized room sets
                          //     tb[3] (the run is then repeated with worst-case room)
  int32_t *cand_c;        // start states of the retained candidates, by position:
                          //   (layer << SD_CAND_SHIFT) | slot on the layer
  int64_t *cand_B;        // their scalar branch costs B(c,b)
  int64_t *Ext;           // N   exterior suffix values (Sec. 5 final-column exterior)
  char *mrna, *structure; // n+1 each
  int64_t *tb;            // [0] energy, [1] path cost, [2] traceback status, [3] overflow
  int32_t *tb_stack;      // traceback work list, 4 ints per task
  int32_t tb_cap;         // tasks
  // Layout of the full tables H, V, B, S1, S2 (one entry per state pair,
  // V six entries):
  //   SD_LAYOUT_SPAN   layer pair (i, i+g) of span g at cell D(g) + i, SD_SLOTS
  //                    state-pair slots per cell (the default; the cells of one
  //                    span are contiguous, which suits the span wavefront)
  //   SD_LAYOUT_SQUARE state pair (a, b) at a*N + b (the paper's square arena)
  //   SD_LAYOUT_PACKED state pair (a, b), b on a later layer than a, at
  //                    poff[a] + b - lstart[layer(a)+1] (the paper's forward-
  //                    packed option: no reverse-layer slots)
  int32_t layout;
  int64_t ncell;          // n(n+1)/2
  int32_t maxin;          // stride of the in-edge lists (SD_MAXIN or SD_MAXIN_WIDE)
  int32_t pad3;
  const int64_t *poff;    // N row offsets (SD_LAYOUT_PACKED only)
  int64_t table_cells;    // state-pair entries of each full table
};

#define SD_LAYOUT_SPAN 0
#define SD_LAYOUT_SQUARE 1
#define SD_LAYOUT_PACKED 2

// Host entry points implemented in sd_kernels.cu.
#ifdef __cplusplus
extern "C" {
#endif
// Designs in device order must have non-increasing n (ns[d] = designs[d].n);
// d_cpre[d] = sum over d' < d of (ns[d'] + 1), count + 1 entries on the device.
// events: NULL or four cudaEvent_t recorded before the fill, after the fill,
// after the exterior pass and after the traceback, on `stream`.
// group: threads per layer pair in the fill (8, 16 or 32).
int sd_k_run(const SdDesign *d_designs, int count, const int *ns, const int32_t *d_cpre,
             const SdParams *d_params, void *stream, int64_t *launches, void *const *events,
             int group);
int sd_k_count_ops(const SdDesign *d_designs, int count, const int *ns, const int32_t *d_cpre,
                   const SdParams *d_params, unsigned long long *d_ops, void *stream, int group);
int sd_k_clear(const SdDesign *h_designs, const SdDesign *d_designs, int count, void *stream);
// host helpers of sd_host.cpp used by the fixed-scratch entry point
struct sd_energy;
char sd_internal_translate(int x, int y, int z);
int64_t sd_internal_codon_fx(double lambda, double w);
int sd_internal_range_check(const struct sd_energy *E, int n, double qmax_sum);
const SdParams *sd_internal_device_params(const struct sd_energy *E);
int sd_internal_on_energy_device(const struct sd_energy *E);  // 1 iff current device == E's
int32_t sd_internal_hairpin_len(const struct sd_energy *E, int L);
// flat edge lists (fo, fi: E entries each; fo_off, fi_off: N+1) from the
// per-state lists
void sd_internal_flatten(int N, const SdEdge *out, const uint8_t *out_cnt, const SdEdge *in,
                         const uint8_t *in_cnt, int maxin, SdFlatEdge *fo, int32_t *fo_off,
                         SdFlatEdge *fi, int32_t *fi_off);
int sd_k_count(const SdDesign *d_designs, int count, int64_t *d_out, void *stream);
int sd_k_retention(const SdDesign *d_designs, int item, int32_t *d_hist, int ncodons,
                   void *stream);
// the same entry points of the wide instance (layers of up to SD_W_WIDE states)
int sd_k_run_wide(const SdDesign *d_designs, int count, const int *ns, const int32_t *d_cpre,
                  const SdParams *d_params, void *stream, int64_t *launches,
                  void *const *events, int group);
int sd_k_count_ops_wide(const SdDesign *d_designs, int count, const int *ns,
                        const int32_t *d_cpre, const SdParams *d_params,
                        unsigned long long *d_ops, void *stream, int group);
int sd_k_count_wide(const SdDesign *d_designs, int count, int64_t *d_out, void *stream);
int sd_k_retention_wide(const SdDesign *d_designs, int item, int32_t *d_hist, int ncodons,
                        void *stream);
#ifdef __cplusplus
}
#endif
