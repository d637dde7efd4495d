/*
 * sd_oracle.c -- plain, slow, dense CPU oracle for exact codon-lattice design.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code with the CUDA path (own parameter parser, own genetic code, own
 * lattice builder, own loop energies, own traceback).
 *
 * What it computes (paper: Sec. 3 Eq. 1 and Sec. 4.1):
 *   F*(p, lambda) = min over synonymous mRNAs r and structures S of
 *                   E_T04,d0(r, S) + lambda' C(r),     lambda' = 100 lambda,
 * over the layered weighted codon DFA of Sec. 3 (-log w on the 3rd codon edge),
 * with the *unsparsified* dense multiloop recurrences (dense2), (partitionable)
 * and (dense1) of Sec. 4.1, evaluated span by span on square N x N tables
 * (the span order of Algorithm 1 without the candidate restriction).
 * Candidate sets C_b (Eq. candidates) are computed from the dense tables by
 * their definition B(c,b) < P_D(c,b) so that tests can compare them.
 *
 * Arithmetic is exact: every DP value is an int64 in units of
 * 2^-32 x 0.01 kcal/mol (energies E*2^32, codon costs
 * round_half_even(lambda' * (-ln w) * 2^32)), so the dense and sparse
 * recurrences agree exactly (Thm. 1 holds in integer arithmetic).
 * +infinity is ORC_INF and every addition is guarded explicitly.
 *
 * Energy model (Sec. 3: Turner-2004 dangle-0, special tri/tetra/hexaloops,
 * lonely pairs, min hairpin 3, at most 30 unpaired nt per bulge/internal loop):
 * the ViennaRNA-style dangle-0 decomposition, read as follows
 *   hairpin L=3      : hairpin[3] + AU(t)
 *   hairpin L>=4     : hairpin[L] + mismatchH[t][x_{i+1}][x_{j-1}]
 *   hairpin L>30     : hairpin[30] + (int)(lxc * ln(L/30)) (+ mismatch)
 *   special (L=3,4,6): the listed value is the total hairpin energy
 *   stack            : stack[t][s]           s = inner pair seen from the loop
 *   bulge 1          : bulge[1] + stack[t][s]
 *   bulge l>1        : bulge[l] + AU(t) + AU(s)
 *   1x1 / 1x2 / 2x2  : int11 / int21 / int22 (2x1 by rotation of int21)
 *   1xn (n>2)        : interior[l] + min(MAXNINIO, ninio|l1-l2|) + mm1n both pairs
 *   2x3 / 3x2        : interior[5] + ninio + mm23 both pairs
 *   other            : interior[l] + min(MAXNINIO, ninio|l1-l2|) + mmI both pairs
 *   multiloop        : closing ML_closing + ML_intern + AU(t); branch
 *                      ML_intern + AU(t); unpaired base ML_base
 *   exterior         : AU(t) per branch; unpaired bases cost no energy.
 * Codon cost lambda' q(e) is charged on every edge exactly once.
 *
 * Canonical tie-break (the paper leaves it open, Sec. 4.2 proof: "A tie causes
 * no difficulty and need not be stored"): first attaining option in the fixed
 * orders written at each trace_* function below.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF ((int64_t)1 << 62)
#define FX(e) ((int64_t)(e) * (int64_t)4294967296LL) /* energy -> fixed point */
#define MAXSPECIAL 256

/* ------------------------------------------------------------------ */
/* parameters                                                           */
/* ------------------------------------------------------------------ */
typedef struct {
  int stack[6][6];
  int mmH[6][4][4], mmI[6][4][4], mm1n[6][4][4], mm23[6][4][4];
  int int11[6][6][4][4];
  int int21[6][6][4][4][4];
  int int22[6][6][4][4][4][4];
  int hairpin[31], bulge[31], interior[31];
  int au[6];
  int ninio, maxninio, mlclosing, mlintern, mlbase;
  double lxc;
  int nspecial[3];                /* tri (5 nt), tetra (6 nt), hexa (8 nt) */
  char special_seq[3][MAXSPECIAL][9];
  int special_e[3][MAXSPECIAL];
} OParams;

static int read_block(FILE *f, const char *name, int *dst, int count) {
  char word[64];
  int n;
  if (fscanf(f, "%63s %d", word, &n) != 2) return -1;
  if (strcmp(word, name) != 0 || n != count) return -1;
  for (int k = 0; k < count; k++)
    if (fscanf(f, "%d", &dst[k]) != 1) return -1;
  return 0;
}

static int load_params(const char *path, OParams *P) {
  FILE *f = fopen(path, "r");
  if (!f) return -1;
  char word[64];
  int ver = 0, rc = 0;
  memset(P, 0, sizeof(*P));
  if (fscanf(f, "%63s %d", word, &ver) != 2 || strcmp(word, "SDENERGY") || ver != 1) rc = -1;
  if (!rc) rc = read_block(f, "stack", &P->stack[0][0], 36);
  if (!rc) rc = read_block(f, "mismatch_hairpin", &P->mmH[0][0][0], 96);
  if (!rc) rc = read_block(f, "mismatch_interior", &P->mmI[0][0][0], 96);
  if (!rc) rc = read_block(f, "mismatch_interior_1n", &P->mm1n[0][0][0], 96);
  if (!rc) rc = read_block(f, "mismatch_interior_23", &P->mm23[0][0][0], 96);
  if (!rc) rc = read_block(f, "int11", &P->int11[0][0][0][0], 576);
  if (!rc) rc = read_block(f, "int21", &P->int21[0][0][0][0][0], 2304);
  if (!rc) rc = read_block(f, "int22", &P->int22[0][0][0][0][0][0], 9216);
  if (!rc) rc = read_block(f, "hairpin", P->hairpin, 31);
  if (!rc) rc = read_block(f, "bulge", P->bulge, 31);
  if (!rc) rc = read_block(f, "interior", P->interior, 31);
  if (!rc) rc = read_block(f, "terminal_au", P->au, 6);
  if (!rc) rc = read_block(f, "ninio", &P->ninio, 1);
  if (!rc) rc = read_block(f, "max_ninio", &P->maxninio, 1);
  if (!rc) rc = read_block(f, "ml_closing", &P->mlclosing, 1);
  if (!rc) rc = read_block(f, "ml_intern", &P->mlintern, 1);
  if (!rc) rc = read_block(f, "ml_base", &P->mlbase, 1);
  if (!rc && (fscanf(f, "%63s %lf", word, &P->lxc) != 2 || strcmp(word, "lxc"))) rc = -1;
  const char *names[3] = {"triloop", "tetraloop", "hexaloop"};
  const int lens[3] = {5, 6, 8};
  for (int s = 0; s < 3 && !rc; s++) {
    int n;
    if (fscanf(f, "%63s %d", word, &n) != 2 || strcmp(word, names[s]) || n < 0 ||
        n > MAXSPECIAL) {
      rc = -1;
      break;
    }
    P->nspecial[s] = n;
    for (int k = 0; k < n && !rc; k++) {
      char seq[64];
      if (fscanf(f, "%63s %d", seq, &P->special_e[s][k]) != 2 || (int)strlen(seq) != lens[s])
        rc = -1;
      else
        strcpy(P->special_seq[s][k], seq);
    }
  }
  fclose(f);
  return rc;
}

/* ------------------------------------------------------------------ */
/* nucleotides, pairs, genetic code                                     */
/* ------------------------------------------------------------------ */
static const char NT[4] = {'A', 'C', 'G', 'U'};
/* oriented pair types: AU CG GC UA GU UG */
static int pair_type(int x, int y) {
  if (x == 0 && y == 3) return 0;
  if (x == 1 && y == 2) return 1;
  if (x == 2 && y == 1) return 2;
  if (x == 3 && y == 0) return 3;
  if (x == 2 && y == 3) return 4;
  if (x == 3 && y == 2) return 5;
  return -1;
}
static const int PAIR5[6] = {0, 1, 2, 3, 2, 3};
static const int PAIR3[6] = {3, 2, 1, 0, 3, 2};
static int rev_type(int t) { return pair_type(PAIR3[t], PAIR5[t]); }

/* The standard genetic code, written out codon by codon (ACGU order). */
static char amino_of_codon(int x, int y, int z) {
  static const char *code =
      /* AAx */ "KNKN" /* ACx */ "TTTT" /* AGx */ "RSRS" /* AUx */ "IIMI"
      /* CAx */ "QHQH" /* CCx */ "PPPP" /* CGx */ "RRRR" /* CUx */ "LLLL"
      /* GAx */ "EDED" /* GCx */ "AAAA" /* GGx */ "GGGG" /* GUx */ "VVVV"
      /* UAx */ "*Y*Y" /* UCx */ "SSSS" /* UGx */ "*CWC" /* UUx */ "LFLF";
  return code[16 * x + 4 * y + z];
}

/* ------------------------------------------------------------------ */
/* lattice                                                              */
/* ------------------------------------------------------------------ */
typedef struct {
  int from, to, label;
  int64_t cost;
} OEdge;

typedef struct {
  int n;             /* number of layers - 1 (nucleotides) */
  int N;             /* states */
  int *layer;        /* layer of each state */
  int *lstart;       /* first state of each layer, lstart[n+1] = N */
  int E;
  OEdge *edges;
  int *out_off, *out_idx; /* out-edges per state, by label */
  int *in_off, *in_idx;   /* in-edges per state, by (label, from) */
  int s, t;
} OLattice;

static void lattice_free(OLattice *L) {
  free(L->layer); free(L->lstart); free(L->edges);
  free(L->out_off); free(L->out_idx); free(L->in_off); free(L->in_idx);
  memset(L, 0, sizeof(*L));
}

static OLattice *g_sort_lattice;
static int cmp_out(const void *a, const void *b) {
  const OEdge *x = &g_sort_lattice->edges[*(const int *)a], *y = &g_sort_lattice->edges[*(const int *)b];
  if (x->from != y->from) return x->from - y->from;
  return x->label - y->label;
}
static int cmp_in(const void *a, const void *b) {
  const OEdge *x = &g_sort_lattice->edges[*(const int *)a], *y = &g_sort_lattice->edges[*(const int *)b];
  if (x->to != y->to) return x->to - y->to;
  if (x->label != y->label) return x->label - y->label;
  return x->from - y->from;
}

static void lattice_index(OLattice *L) {
  int N = L->N, E = L->E;
  L->out_off = calloc(N + 1, sizeof(int));
  L->in_off = calloc(N + 1, sizeof(int));
  L->out_idx = malloc(sizeof(int) * (E > 0 ? E : 1));
  L->in_idx = malloc(sizeof(int) * (E > 0 ? E : 1));
  for (int e = 0; e < E; e++) { L->out_idx[e] = e; L->in_idx[e] = e; }
  g_sort_lattice = L;
  qsort(L->out_idx, E, sizeof(int), cmp_out);
  qsort(L->in_idx, E, sizeof(int), cmp_in);
  for (int e = 0; e < E; e++) { L->out_off[L->edges[e].from + 1]++; L->in_off[L->edges[e].to + 1]++; }
  for (int v = 0; v < N; v++) { L->out_off[v + 1] += L->out_off[v]; L->in_off[v + 1] += L->in_off[v]; }
}

/* Fixed-point codon cost: round_half_even(lambda' * (-ln w) * 2^32). */
static int64_t codon_cost_fx(double lambda, double w) {
  double lam100 = 100.0 * lambda;
  double q = -log(w);
  double x = lam100 * q;
  return (int64_t)llrint(ldexp(x, 32));
}

/* Codon trie per amino acid (Sec. 3): one state per codon boundary, one state
 * per distinct first nucleotide and per distinct 2-prefix; the whole -ln w on
 * the third edge.  States inside a layer are numbered by their codon prefix in
 * ACGU order. Returns 0, or -1 on invalid input. */
static int build_codon_lattice(const char *protein, const double *w, double lambda, OLattice *L) {
  memset(L, 0, sizeof(*L));
  int A = (int)strlen(protein);
  for (int k = 0; k < A; k++)
    if (protein[k] == '*' && k != A - 1) return -1;
  int n = 3 * A;
  int cap = 8 * A + 2;
  L->n = n;
  L->layer = malloc(sizeof(int) * cap);
  L->lstart = malloc(sizeof(int) * (n + 2));
  L->edges = malloc(sizeof(OEdge) * (12 * A + 1)); /* <= 10 edges per codon position */
  int N = 0, E = 0;
  L->lstart[0] = 0;
  L->layer[N++] = 0; /* source */
  int boundary = 0;
  for (int k = 0; k < A; k++) {
    char aa = protein[k];
    int cod[64][3], nc = 0;
    double wmax = 0.0;
    for (int x = 0; x < 4; x++)
      for (int y = 0; y < 4; y++)
        for (int z = 0; z < 4; z++)
          if (amino_of_codon(x, y, z) == aa) {
            cod[nc][0] = x; cod[nc][1] = y; cod[nc][2] = z; nc++;
            double ww = w[16 * x + 4 * y + z];
            if (!(ww > 0.0 && ww <= 1.0)) { lattice_free(L); return -1; }
            if (ww > wmax) wmax = ww;
          }
    if (nc == 0 || wmax != 1.0) { lattice_free(L); return -1; }
    /* layer 3k+1: distinct first nucleotides, ascending */
    int first_id[4] = {-1, -1, -1, -1};
    L->lstart[3 * k + 1] = N;
    for (int x = 0; x < 4; x++)
      for (int c = 0; c < nc; c++)
        if (cod[c][0] == x) { first_id[x] = N; L->layer[N++] = 3 * k + 1; break; }
    /* layer 3k+2: distinct prefixes, ascending */
    int pre_id[4][4];
    for (int x = 0; x < 4; x++) for (int y = 0; y < 4; y++) pre_id[x][y] = -1;
    L->lstart[3 * k + 2] = N;
    for (int x = 0; x < 4; x++)
      for (int y = 0; y < 4; y++)
        for (int c = 0; c < nc; c++)
          if (cod[c][0] == x && cod[c][1] == y) { pre_id[x][y] = N; L->layer[N++] = 3 * k + 2; break; }
    /* next boundary */
    L->lstart[3 * k + 3] = N;
    int nb = N;
    L->layer[N++] = 3 * k + 3;
    for (int x = 0; x < 4; x++)
      if (first_id[x] >= 0) { OEdge e = {boundary, first_id[x], x, 0}; L->edges[E++] = e; }
    for (int x = 0; x < 4; x++)
      for (int y = 0; y < 4; y++)
        if (pre_id[x][y] >= 0) { OEdge e = {first_id[x], pre_id[x][y], y, 0}; L->edges[E++] = e; }
    for (int c = 0; c < nc; c++) {
      int x = cod[c][0], y = cod[c][1], z = cod[c][2];
      OEdge e = {pre_id[x][y], nb, z, codon_cost_fx(lambda, w[16 * x + 4 * y + z])};
      L->edges[E++] = e;
    }
    boundary = nb;
  }
  L->lstart[n + 1] = N;
  L->N = N;
  L->E = E;
  L->s = 0;
  L->t = N - 1;
  lattice_index(L);
  return 0;
}

/* A single fixed RNA sequence as a width-1 lattice with zero edge costs. */
static int build_rna_lattice(const char *rna, OLattice *L) {
  memset(L, 0, sizeof(*L));
  int n = (int)strlen(rna);
  L->n = n;
  L->N = n + 1;
  L->layer = malloc(sizeof(int) * (n + 1));
  L->lstart = malloc(sizeof(int) * (n + 2));
  L->edges = malloc(sizeof(OEdge) * (n + 1));
  for (int k = 0; k <= n; k++) { L->layer[k] = k; L->lstart[k] = k; }
  L->lstart[n + 1] = n + 1;
  for (int k = 0; k < n; k++) {
    int lab = -1;
    for (int c = 0; c < 4; c++) if (rna[k] == NT[c]) lab = c;
    if (lab < 0) { lattice_free(L); return -1; }
    OEdge e = {k, k + 1, lab, 0};
    L->edges[k] = e;
  }
  L->E = n;
  L->s = 0;
  L->t = n;
  lattice_index(L);
  return 0;
}

/* ------------------------------------------------------------------ */
/* forbidden motifs (Sec. 3): codon DFA x Aho-Corasick automaton         */
/* ------------------------------------------------------------------ */
#define MAXPRE 2048
typedef struct {
  int n;                    /* matcher states = distinct motif prefixes  */
  char pre[MAXPRE][33];     /* ordered by (length, sequence)             */
  int go[MAXPRE][4];        /* longest suffix of pre+c that is a prefix  */
  int bad[MAXPRE];          /* pre ends with a motif                     */
} Matcher;

static int pre_cmp(const void *a, const void *b) {
  const char *x = (const char *)a, *y = (const char *)b;
  size_t lx = strlen(x), ly = strlen(y);
  if (lx != ly) return lx < ly ? -1 : 1;
  return strcmp(x, y);
}

static int pre_find(const Matcher *M, const char *s) {
  for (int k = 0; k < M->n; k++)
    if (strcmp(M->pre[k], s) == 0) return k;
  return -1;
}

/* motifs: comma-separated strings over ACGU; returns 0 or -1 */
static int matcher_build(const char *motifs, Matcher *M) {
  char mot[64][33];
  int nm = 0;
  const char *p = motifs;
  while (*p) {
    int len = 0;
    while (p[len] && p[len] != ',') len++;
    if (len == 0 || len > 32 || nm >= 64) return -1;
    memcpy(mot[nm], p, len);
    mot[nm][len] = 0;
    for (int k = 0; k < len; k++)
      if (!strchr("ACGU", mot[nm][k])) return -1;
    nm++;
    p += len;
    if (*p == ',') p++;
  }
  M->n = 0;
  M->pre[M->n++][0] = 0;
  for (int k = 0; k < nm; k++)
    for (int l = 1; l <= (int)strlen(mot[k]); l++) {
      char buf[33];
      memcpy(buf, mot[k], l);
      buf[l] = 0;
      if (pre_find(M, buf) < 0) {
        if (M->n >= MAXPRE) return -1;
        strcpy(M->pre[M->n++], buf);
      }
    }
  qsort(M->pre, M->n, sizeof(M->pre[0]), pre_cmp);
  for (int k = 0; k < M->n; k++) {
    M->bad[k] = 0;
    size_t lk = strlen(M->pre[k]);
    for (int q = 0; q < nm; q++) {
      size_t lq = strlen(mot[q]);
      if (lk >= lq && strcmp(M->pre[k] + lk - lq, mot[q]) == 0) M->bad[k] = 1;
    }
    for (int c = 0; c < 4; c++) {
      char t[40];
      strcpy(t, M->pre[k]);
      size_t lt = strlen(t);
      t[lt] = NT[c];
      t[lt + 1] = 0;
      const char *u = t;
      int id;
      while ((id = pre_find(M, u)) < 0) u++;
      M->go[k][c] = id;
    }
  }
  return 0;
}

typedef struct { int q, m; } PState;
static int pstate_cmp(const void *a, const void *b) {
  const PState *x = (const PState *)a, *y = (const PState *)b;
  if (x->q != y->q) return x->q - y->q;
  return x->m - y->m;
}

/* Product of a layered lattice with the matcher: states (q, m) reachable
 * without entering a bad m, the last layer merged into one sink, trimmed to
 * states reaching the sink; layer by layer, (q, m) order inside a layer.
 * Returns 0, -3 for an empty language, -1 on failure. */
static int motif_product(const OLattice *L0, const Matcher *M, OLattice *L) {
  int n = L0->n;
  /* states of the product per layer */
  PState **lay = calloc(n + 1, sizeof(PState *));
  int *cnt = calloc(n + 1, sizeof(int)), *cap = calloc(n + 1, sizeof(int));
  typedef struct { int l, a, b, label; int64_t cost; } PEdge; /* a, b: index in layer */
  PEdge *pe = NULL;
  int npe = 0, cpe = 0, rc = 0;
  lay[0] = malloc(sizeof(PState));
  lay[0][0].q = L0->s;
  lay[0][0].m = 0;
  cnt[0] = cap[0] = 1;
  for (int l = 0; l < n; l++) {
    /* targets of layer l + 1, then sort them into (q, m) order */
    for (int pass = 0; pass < 2; pass++) {
      for (int a = 0; a < cnt[l]; a++) {
        int q = lay[l][a].q, m = lay[l][a].m;
        for (int k = L0->out_off[q]; k < L0->out_off[q + 1]; k++) {
          const OEdge *e = &L0->edges[L0->out_idx[k]];
          int m2 = M->go[m][e->label];
          if (M->bad[m2]) continue;
          PState t = {e->to, l + 1 == n ? 0 : m2};
          int b = -1;
          for (int x = 0; x < cnt[l + 1]; x++)
            if (lay[l + 1][x].q == t.q && lay[l + 1][x].m == t.m) { b = x; break; }
          if (pass == 0) {
            if (b < 0) {
              if (cnt[l + 1] == cap[l + 1]) {
                cap[l + 1] = cap[l + 1] ? 2 * cap[l + 1] : 8;
                lay[l + 1] = realloc(lay[l + 1], sizeof(PState) * cap[l + 1]);
              }
              lay[l + 1][cnt[l + 1]++] = t;
            }
          } else {
            if (npe == cpe) {
              cpe = cpe ? 2 * cpe : 64;
              pe = realloc(pe, sizeof(PEdge) * cpe);
            }
            PEdge x = {l, a, b, e->label, e->cost};
            pe[npe++] = x;
          }
        }
      }
      if (pass == 0 && cnt[l + 1] > 1) qsort(lay[l + 1], cnt[l + 1], sizeof(PState), pstate_cmp);
    }
  }
  if (cnt[n] == 0) {
    rc = -3;
  } else {
    /* backward trim */
    int **live = calloc(n + 1, sizeof(int *));
    for (int l = 0; l <= n; l++) live[l] = calloc(cnt[l] > 0 ? cnt[l] : 1, sizeof(int));
    live[n][0] = 1;
    for (int l = n - 1; l >= 0; l--)
      for (int k = 0; k < npe; k++)
        if (pe[k].l == l && live[l + 1][pe[k].b]) live[l][pe[k].a] = 1;
    if (!live[0][0]) {
      rc = -3;
    } else {
      /* renumber */
      int **nid = calloc(n + 1, sizeof(int *));
      int N = 0;
      memset(L, 0, sizeof(*L));
      L->n = n;
      L->lstart = malloc(sizeof(int) * (n + 2));
      int total = 0;
      for (int l = 0; l <= n; l++) total += cnt[l];
      L->layer = malloc(sizeof(int) * (total > 0 ? total : 1));
      for (int l = 0; l <= n; l++) {
        nid[l] = malloc(sizeof(int) * (cnt[l] > 0 ? cnt[l] : 1));
        L->lstart[l] = N;
        for (int a = 0; a < cnt[l]; a++) {
          nid[l][a] = live[l][a] ? N : -1;
          if (live[l][a]) L->layer[N++] = l;
        }
      }
      L->lstart[n + 1] = N;
      L->N = N;
      L->edges = malloc(sizeof(OEdge) * (npe > 0 ? npe : 1));
      int E = 0;
      for (int k = 0; k < npe; k++) {
        int a = nid[pe[k].l][pe[k].a], b = nid[pe[k].l + 1][pe[k].b];
        if (a < 0 || b < 0) continue;
        OEdge e = {a, b, pe[k].label, pe[k].cost};
        L->edges[E++] = e;
      }
      L->E = E;
      L->s = 0;
      L->t = N - 1;
      lattice_index(L);
      for (int l = 0; l <= n; l++) free(nid[l]);
      free(nid);
    }
    for (int l = 0; l <= n; l++) free(live[l]);
    free(live);
  }
  for (int l = 0; l <= n; l++) free(lay[l]);
  free(lay);
  free(cnt);
  free(cap);
  free(pe);
  return rc;
}

/* ------------------------------------------------------------------ */
/* loop energies (integer dcal/mol)                                     */
/* ------------------------------------------------------------------ */
static int hairpin_len_energy(const OParams *P, int L) {
  if (L <= 30) return P->hairpin[L];
  return P->hairpin[30] + (int)(P->lxc * log((double)L / 30.0));
}

/* generic (non-special) hairpin energy of closing pair t, loop length L,
 * first and last loop nucleotides f, l */
static int hairpin_generic(const OParams *P, int t, int L, int f, int l) {
  if (L == 3) return P->hairpin[3] + P->au[t];
  return hairpin_len_energy(P, L) + P->mmH[t][f][l];
}

/* hairpin energy of a complete hairpin sequence seq[0..L+1] (pair + loop) */
static int hairpin_seq_energy(const OParams *P, int t, const int *seq, int L) {
  int s = L == 3 ? 0 : L == 4 ? 1 : L == 6 ? 2 : -1;
  if (s >= 0) {
    char buf[16];
    for (int k = 0; k < L + 2; k++) buf[k] = NT[seq[k]];
    buf[L + 2] = 0;
    for (int k = 0; k < P->nspecial[s]; k++)
      if (strcmp(buf, P->special_seq[s][k]) == 0) return P->special_e[s][k];
  }
  return hairpin_generic(P, t, L, seq[1], seq[L]);
}

/* two-loop energy; t outer pair, ti inner pair (5'->3' as in the sequence),
 * l1/l2 unpaired on the 5'/3' side, xi1 = nt i+1, xp1 = nt p-1,
 * xq1 = nt q+1, xj1 = nt j-1 (only those that exist are read) */
static int twoloop_energy(const OParams *P, int t, int ti, int l1, int l2, int xi1, int xp1,
                          int xq1, int xj1) {
  int s = rev_type(ti);
  if (l1 == 0 && l2 == 0) return P->stack[t][s];
  if (l1 == 0 || l2 == 0) {
    int l = l1 + l2;
    if (l == 1) return P->bulge[1] + P->stack[t][s];
    return P->bulge[l] + P->au[t] + P->au[s];
  }
  if (l1 == 1 && l2 == 1) return P->int11[t][s][xi1][xj1];
  if (l1 == 1 && l2 == 2) return P->int21[t][s][xi1][xq1][xj1];
  if (l1 == 2 && l2 == 1) return P->int21[s][t][xq1][xi1][xp1];
  if (l1 == 2 && l2 == 2) return P->int22[t][s][xi1][xp1][xq1][xj1];
  int d = l1 > l2 ? l1 - l2 : l2 - l1;
  int asym = P->ninio * d < P->maxninio ? P->ninio * d : P->maxninio;
  if (l1 == 1 || l2 == 1)
    return P->interior[l1 + l2] + asym + P->mm1n[t][xi1][xj1] + P->mm1n[s][xq1][xp1];
  if ((l1 == 2 && l2 == 3) || (l1 == 3 && l2 == 2))
    return P->interior[5] + P->ninio + P->mm23[t][xi1][xj1] + P->mm23[s][xq1][xp1];
  return P->interior[l1 + l2] + asym + P->mmI[t][xi1][xj1] + P->mmI[s][xq1][xp1];
}

/* ------------------------------------------------------------------ */
/* the design                                                           */
/* ------------------------------------------------------------------ */
typedef struct orc_design {
  OParams P;
  OLattice L;
  double lambda;
  int64_t *H;   /* N*N min path cost a->b (H[a][a] = 0)              */
  int64_t *V;   /* N*N*6 typed closed values V_t(a,b)                */
  int64_t *Bv;  /* N*N branch interface B(a,b) = min_t V_t + beta_t   */
  int64_t *D1, *D2, *PD; /* N*N dense multiloop values                */
  int64_t *Ext; /* N exterior suffix values                           */
  unsigned char *cand; /* N*N, cand[c*N+b] = 1 iff c in C_b          */
  /* result */
  char *mrna, *structure;
  int32_t energy;
  int64_t path_cost_fx;
  int64_t obj_fx;
  double codon_cost, objective;
  int64_t Z, finite_direct, retained_cells;
  int status; /* 0 ok, 1 traceback failure */
  /* traceback scratch */
  int64_t tb_energy;
} orc_design;

#define IDX(a, b) ((size_t)(a) * (size_t)N + (size_t)(b))

static int64_t add2(int64_t x, int64_t y) { return (x >= ORC_INF || y >= ORC_INF) ? ORC_INF : x + y; }
static int64_t add3(int64_t x, int64_t y, int64_t z) { return add2(add2(x, y), z); }
static int64_t mn(int64_t x, int64_t y) { return x < y ? x : y; }

/* H'(x,y): min path cost x -> y, 0 for x == y, INF when no path */
static int64_t Hp(const orc_design *D, int x, int y) {
  int N = D->L.N;
  if (x == y) return 0;
  if (D->L.layer[y] <= D->L.layer[x]) return ORC_INF;
  return D->H[IDX(x, y)];
}

/* out-edge of x with a given label, or -1 */
static int out_edge(const OLattice *L, int x, int label) {
  for (int k = L->out_off[x]; k < L->out_off[x + 1]; k++)
    if (L->edges[L->out_idx[k]].label == label) return L->out_idx[k];
  return -1;
}

/* --- gap descriptors: the facts a loop energy can see about an unpaired
 *     stretch from state x to state y of length len ------------------- */
typedef struct {
  int first, last; /* first / last nucleotide (len >= 1) */
  int64_t cost;    /* min path cost realising it */
  int e1, e2;      /* len 1: e1; len 2: e1 e2 (explicit path) */
} GapDesc;

/* enumerate descriptors in canonical order: len 0: one; len 1: parallel edges
 * by label; len 2: explicit 2-edge paths by (label1, label2); len >= 3:
 * (first, last) label pairs in lexicographic order with min cost
 * G(x,y,f,l) = min over x->x2 (f), m->y (l) of c + H'(x2,m) + c. */
static int gap_descs(const orc_design *D, int x, int y, int len, GapDesc *out) {
  const OLattice *L = &D->L;
  int n = 0;
  if (len == 0) {
    if (x == y) { GapDesc g = {-1, -1, 0, -1, -1}; out[n++] = g; }
    return n;
  }
  if (len == 1) {
    for (int k = L->out_off[x]; k < L->out_off[x + 1]; k++) {
      const OEdge *e = &L->edges[L->out_idx[k]];
      if (e->to == y) { GapDesc g = {e->label, e->label, e->cost, L->out_idx[k], -1}; out[n++] = g; }
    }
    return n;
  }
  if (len == 2) {
    for (int k = L->out_off[x]; k < L->out_off[x + 1]; k++) {
      const OEdge *e = &L->edges[L->out_idx[k]];
      int m = e->to;
      for (int k2 = L->out_off[m]; k2 < L->out_off[m + 1]; k2++) {
        const OEdge *e2 = &L->edges[L->out_idx[k2]];
        if (e2->to == y) {
          GapDesc g = {e->label, e2->label, e->cost + e2->cost, L->out_idx[k], L->out_idx[k2]};
          out[n++] = g;
        }
      }
    }
    return n;
  }
  for (int f = 0; f < 4; f++) {
    int ex = out_edge(L, x, f);
    if (ex < 0) continue;
    int x2 = L->edges[ex].to;
    for (int l = 0; l < 4; l++) {
      int64_t best = ORC_INF;
      for (int k = L->in_off[y]; k < L->in_off[y + 1]; k++) {
        const OEdge *e = &L->edges[L->in_idx[k]];
        if (e->label != l) continue;
        best = mn(best, add3(L->edges[ex].cost, Hp(D, x2, e->from), e->cost));
      }
      if (best < ORC_INF) { GapDesc g = {f, l, best, ex, -1}; out[n++] = g; }
    }
  }
  return n;
}

/* --- explicit path enumeration for special-length hairpins ---------- */
typedef void (*path_cb)(void *ctx, const int *labels, const int *edges, int len, int64_t cost);
static void enum_paths_rec(const OLattice *L, int x, int y, int left, int *lab, int *edg, int depth,
                           int64_t cost, path_cb cb, void *ctx) {
  if (left == 0) {
    if (x == y) cb(ctx, lab, edg, depth, cost);
    return;
  }
  for (int k = L->out_off[x]; k < L->out_off[x + 1]; k++) {
    const OEdge *e = &L->edges[L->out_idx[k]];
    lab[depth] = e->label;
    edg[depth] = L->out_idx[k];
    enum_paths_rec(L, e->to, y, left - 1, lab, edg, depth + 1, cost + e->cost, cb, ctx);
  }
}

typedef struct {
  const orc_design *D;
  int t;
  int64_t best;
  /* traceback mode */
  int64_t target;
  int found;
  int edges[16];
  int energy;
} HpCtx;

static void hp_cb(void *vctx, const int *lab, const int *edg, int len, int64_t cost) {
  HpCtx *c = (HpCtx *)vctx;
  int seq[16];
  seq[0] = PAIR5[c->t];
  for (int k = 0; k < len; k++) seq[k + 1] = lab[k];
  seq[len + 1] = PAIR3[c->t];
  int e = hairpin_seq_energy(&c->D->P, c->t, seq, len);
  int64_t v = FX(e) + cost;
  if (v < c->best) c->best = v;
  if (!c->found && c->target < ORC_INF && v == c->target) {
    c->found = 1;
    c->energy = e;
    for (int k = 0; k < len; k++) c->edges[k] = edg[k];
  }
}

/* hairpin part of a closed value: pair t, interior path x -> y of L edges */
static int64_t hairpin_min(const orc_design *D, int x, int y, int t, int L) {
  if (L < 3) return ORC_INF;
  if (L == 3 || L == 4 || L == 6) {
    HpCtx c;
    memset(&c, 0, sizeof(c));
    c.D = D; c.t = t; c.best = ORC_INF; c.target = ORC_INF;
    int lab[16], edg[16];
    enum_paths_rec(&D->L, x, y, L, lab, edg, 0, 0, hp_cb, &c);
    return c.best;
  }
  GapDesc g[64];
  int ng = gap_descs(D, x, y, L, g);
  int64_t best = ORC_INF;
  for (int k = 0; k < ng; k++)
    best = mn(best, add2(FX(hairpin_generic(&D->P, t, L, g[k].first, g[k].last)), g[k].cost));
  return best;
}

/* two-loop part: pair t outside, loop region from x (after the 5' nt of the
 * pair) to y (before its 3' nt) */
static int64_t twoloop_min(const orc_design *D, int x, int y, int t) {
  const OLattice *L = &D->L;
  int N = L->N;
  int64_t best = ORC_INF;
  int lx = L->layer[x], ly = L->layer[y];
  GapDesc gl[64], gr[64];
  for (int l = 0; l <= 30; l++)
    for (int l1 = 0; l1 <= l; l1++) {
      int l2 = l - l1;
      int lc = lx + l1, ld = ly - l2;
      if (ld - lc < 5) continue; /* the inner pair needs span >= 5 */
      for (int c = L->lstart[lc]; c < L->lstart[lc + 1]; c++)
        for (int d = L->lstart[ld]; d < L->lstart[ld + 1]; d++) {
          int ngl = gap_descs(D, x, c, l1, gl);
          if (!ngl) continue;
          int ngr = gap_descs(D, d, y, l2, gr);
          if (!ngr) continue;
          for (int ti = 0; ti < 6; ti++) {
            int64_t v = D->V[IDX(c, d) * 6 + ti];
            if (v >= ORC_INF) continue;
            for (int a = 0; a < ngl; a++)
              for (int b = 0; b < ngr; b++) {
                int e = twoloop_energy(&D->P, t, ti, l1, l2, gl[a].first, gl[a].last, gr[b].first,
                                       gr[b].last);
                best = mn(best, add3(v, FX(e), gl[a].cost + gr[b].cost));
              }
          }
        }
    }
  return best;
}

static int64_t mlclose_fx(const OParams *P, int t) { return FX(P->mlclosing + P->mlintern + P->au[t]); }
static int64_t beta_fx(const OParams *P, int t) { return FX(P->mlintern + P->au[t]); }
static int64_t u_fx(const orc_design *D, const OEdge *e) { return e->cost + FX(D->P.mlbase); }

/* V_t(a,b) for span >= 5 (Sec. 4.1): the first edge of a with label 5'(t),
 * any last edge into b with label 3'(t), closed by hairpin / two-loop /
 * multiloop. */
static int64_t closed_value(const orc_design *D, int a, int b, int t) {
  const OLattice *L = &D->L;
  int N = L->N;
  int ex = out_edge(L, a, PAIR5[t]);
  if (ex < 0) return ORC_INF;
  int a1 = L->edges[ex].to;
  int64_t best = ORC_INF;
  for (int k = L->in_off[b]; k < L->in_off[b + 1]; k++) {
    const OEdge *ey = &L->edges[L->in_idx[k]];
    if (ey->label != PAIR3[t]) continue;
    int b1 = ey->from;
    int Ln = L->layer[b1] - L->layer[a1];
    int64_t base = L->edges[ex].cost + ey->cost;
    best = mn(best, add2(base, hairpin_min(D, a1, b1, t, Ln)));
    best = mn(best, add2(base, twoloop_min(D, a1, b1, t)));
    if (Ln >= 1) best = mn(best, add3(base, mlclose_fx(&D->P, t), D->D2[IDX(a1, b1)]));
  }
  return best;
}

static int g_threads = 1; /* threads filling one span (orc_set_threads) */

static void fill(orc_design *D) {
  OLattice *L = &D->L;
  int N = L->N, n = L->n;
  size_t NN = (size_t)N * N;
  D->H = malloc(sizeof(int64_t) * NN);
  D->V = malloc(sizeof(int64_t) * NN * 6);
  D->Bv = malloc(sizeof(int64_t) * NN);
  D->D1 = malloc(sizeof(int64_t) * NN);
  D->D2 = malloc(sizeof(int64_t) * NN);
  D->PD = malloc(sizeof(int64_t) * NN);
  D->cand = calloc(NN, 1);
  D->Ext = malloc(sizeof(int64_t) * N);
  for (size_t k = 0; k < NN; k++) { D->H[k] = D->Bv[k] = D->D1[k] = D->D2[k] = D->PD[k] = ORC_INF; }
  for (size_t k = 0; k < NN * 6; k++) D->V[k] = ORC_INF;
  for (int g = 1; g <= n; g++)
    /* the cells of one span depend only on smaller spans (Algorithm 1), so
       its layer pairs may be filled by several threads (one by default) */
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
    for (int i = 0; i <= n - g; i++) {
      int j = i + g;
      for (int a = L->lstart[i]; a < L->lstart[i + 1]; a++)
        for (int b = L->lstart[j]; b < L->lstart[j + 1]; b++) {
          size_t ab = IDX(a, b);
          /* gap path cost */
          int64_t h = ORC_INF;
          for (int k = L->in_off[b]; k < L->in_off[b + 1]; k++) {
            const OEdge *e = &L->edges[L->in_idx[k]];
            h = mn(h, add2(Hp(D, a, e->from), e->cost));
          }
          D->H[ab] = h;
          /* typed closed values and the branch interface, Eq. (branch) */
          int64_t Bab = ORC_INF;
          if (g >= 5)
            for (int t = 0; t < 6; t++) {
              int64_t v = closed_value(D, a, b, t);
              D->V[ab * 6 + t] = v;
              Bab = mn(Bab, add2(v, beta_fx(&D->P, t)));
            }
          D->Bv[ab] = Bab;
          /* Eq. (dense2) */
          int64_t d2 = ORC_INF;
          for (int k = L->in_off[b]; k < L->in_off[b + 1]; k++) {
            const OEdge *e = &L->edges[L->in_idx[k]];
            if (L->layer[e->from] > i) d2 = mn(d2, add2(D->D2[IDX(a, e->from)], u_fx(D, e)));
          }
          for (int c = L->lstart[i + 1]; c < L->lstart[j]; c++)
            d2 = mn(d2, add2(D->D1[IDX(a, c)], D->Bv[IDX(c, b)]));
          D->D2[ab] = d2;
          /* Eq. (partitionable) */
          int64_t pd = d2;
          for (int k = L->out_off[a]; k < L->out_off[a + 1]; k++) {
            const OEdge *e = &L->edges[L->out_idx[k]];
            if (L->layer[e->to] < j) pd = mn(pd, add2(u_fx(D, e), D->D1[IDX(e->to, b)]));
          }
          for (int k = L->in_off[b]; k < L->in_off[b + 1]; k++) {
            const OEdge *e = &L->edges[L->in_idx[k]];
            if (L->layer[e->from] > i) pd = mn(pd, add2(D->D1[IDX(a, e->from)], u_fx(D, e)));
          }
          D->PD[ab] = pd;
          /* Eq. (dense1) and Eq. (candidates) */
          D->D1[ab] = mn(Bab, pd);
          D->cand[ab] = (Bab < pd) ? 1 : 0;
        }
    }
  /* exterior suffix values at the final state (Sec. 5) */
  for (int v = 0; v < N; v++) D->Ext[v] = ORC_INF;
  D->Ext[L->t] = 0;
  for (int k = n - 1; k >= 0; k--)
    for (int a = L->lstart[k]; a < L->lstart[k + 1]; a++) {
      int64_t best = ORC_INF;
      for (int q = L->out_off[a]; q < L->out_off[a + 1]; q++) {
        const OEdge *e = &L->edges[L->out_idx[q]];
        best = mn(best, add2(e->cost, D->Ext[e->to]));
      }
      for (int b = L->lstart[k + 1]; b < N; b++)
        for (int t = 0; t < 6; t++)
          best = mn(best, add3(D->V[IDX(a, b) * 6 + t], FX(D->P.au[t]), D->Ext[b]));
      D->Ext[a] = best;
    }
  /* counters */
  D->Z = D->finite_direct = D->retained_cells = 0;
  for (size_t k = 0; k < NN; k++) {
    if (D->Bv[k] < ORC_INF) D->finite_direct++;
    if (D->cand[k]) D->Z++;
    if (D->D1[k] < ORC_INF) D->retained_cells++;
    if (D->D2[k] < ORC_INF) D->retained_cells++;
    for (int t = 0; t < 6; t++)
      if (D->V[k * 6 + t] < ORC_INF) D->retained_cells++;
  }
  D->retained_cells += D->Z;
}

/* ------------------------------------------------------------------ */
/* canonical traceback                                                  */
/* ------------------------------------------------------------------ */
static int tb_fail;
static void emit_edge(orc_design *D, int e) {
  const OEdge *ed = &D->L.edges[e];
  int pos = D->L.layer[ed->from];
  if (D->mrna[pos] != '?') tb_fail = 1;
  D->mrna[pos] = NT[ed->label];
  D->path_cost_fx += ed->cost;
}

/* canonical min-cost gap path: greedy, out-edges in label order */
static void trace_gap(orc_design *D, int x, int y) {
  const OLattice *L = &D->L;
  while (x != y) {
    int64_t v = Hp(D, x, y);
    int moved = 0;
    for (int k = L->out_off[x]; k < L->out_off[x + 1]; k++) {
      const OEdge *e = &L->edges[L->out_idx[k]];
      if (L->layer[e->to] > L->layer[y]) continue;
      if (add2(e->cost, Hp(D, e->to, y)) == v) {
        emit_edge(D, L->out_idx[k]);
        x = e->to;
        moved = 1;
        break;
      }
    }
    if (!moved) { tb_fail = 1; return; }
  }
}

/* realise a gap descriptor from x to y of length len */
static void trace_desc(orc_design *D, int y, int len, const GapDesc *g) {
  const OLattice *L = &D->L;
  if (len == 0) return;
  if (len == 1) { emit_edge(D, g->e1); return; }
  if (len == 2) { emit_edge(D, g->e1); emit_edge(D, g->e2); return; }
  int x2 = L->edges[g->e1].to;
  for (int k = L->in_off[y]; k < L->in_off[y + 1]; k++) {
    const OEdge *e = &L->edges[L->in_idx[k]];
    if (e->label != g->last) continue;
    if (add3(L->edges[g->e1].cost, Hp(D, x2, e->from), e->cost) == g->cost) {
      emit_edge(D, g->e1);
      trace_gap(D, x2, e->from);
      emit_edge(D, L->in_idx[k]);
      return;
    }
  }
  tb_fail = 1;
}

static void trace_D1(orc_design *D, int a, int b);
static void trace_D2(orc_design *D, int a, int b);

static void set_pair(orc_design *D, int i, int j) {
  if (D->structure[i] != '.' || D->structure[j] != '.') tb_fail = 1;
  D->structure[i] = '(';
  D->structure[j] = ')';
}

/* V_t(a,b): for each last edge (in-edge order: label, from), try hairpin
 * (special lengths: interior paths in lexicographic label order; otherwise
 * (first,last) descriptors in lexicographic order), then two-loops in
 * (l1+l2, l1, c, d, inner type, left descriptor, right descriptor) order,
 * then the multiloop. */
static void trace_V(orc_design *D, int a, int b, int t) {
  const OLattice *L = &D->L;
  int N = L->N;
  int64_t v = D->V[IDX(a, b) * 6 + t];
  int ex = out_edge(L, a, PAIR5[t]);
  if (ex < 0 || v >= ORC_INF) { tb_fail = 1; return; }
  int a1 = L->edges[ex].to;
  set_pair(D, L->layer[a], L->layer[b] - 1);
  for (int k = L->in_off[b]; k < L->in_off[b + 1]; k++) {
    const OEdge *ey = &L->edges[L->in_idx[k]];
    if (ey->label != PAIR3[t]) continue;
    int eyi = L->in_idx[k];
    int b1 = ey->from;
    int Ln = L->layer[b1] - L->layer[a1];
    int64_t base = L->edges[ex].cost + ey->cost;
    /* hairpin */
    if (Ln >= 3) {
      if (Ln == 3 || Ln == 4 || Ln == 6) {
        HpCtx c;
        memset(&c, 0, sizeof(c));
        c.D = D; c.t = t; c.best = ORC_INF; c.target = v - base;
        int lab[16], edg[16];
        enum_paths_rec(L, a1, b1, Ln, lab, edg, 0, 0, hp_cb, &c);
        if (c.found) {
          emit_edge(D, ex);
          for (int q = 0; q < Ln; q++) emit_edge(D, c.edges[q]);
          emit_edge(D, eyi);
          D->tb_energy += c.energy;
          return;
        }
      } else {
        GapDesc g[64];
        int ng = gap_descs(D, a1, b1, Ln, g);
        for (int q = 0; q < ng; q++) {
          int e = hairpin_generic(&D->P, t, Ln, g[q].first, g[q].last);
          if (add3(base, FX(e), g[q].cost) == v) {
            emit_edge(D, ex);
            trace_desc(D, b1, Ln, &g[q]);
            emit_edge(D, eyi);
            D->tb_energy += e;
            return;
          }
        }
      }
    }
    /* two-loops */
    int lx = L->layer[a1], ly = L->layer[b1];
    GapDesc gl[64], gr[64];
    for (int l = 0; l <= 30; l++)
      for (int l1 = 0; l1 <= l; l1++) {
        int l2 = l - l1;
        int lc = lx + l1, ld = ly - l2;
        if (ld - lc < 5) continue;
        for (int c = L->lstart[lc]; c < L->lstart[lc + 1]; c++)
          for (int d = L->lstart[ld]; d < L->lstart[ld + 1]; d++) {
            int ngl = gap_descs(D, a1, c, l1, gl);
            int ngr = gap_descs(D, d, b1, l2, gr);
            for (int ti = 0; ti < 6; ti++) {
              int64_t vi = D->V[IDX(c, d) * 6 + ti];
              if (vi >= ORC_INF) continue;
              for (int p = 0; p < ngl; p++)
                for (int r = 0; r < ngr; r++) {
                  int e = twoloop_energy(&D->P, t, ti, l1, l2, gl[p].first, gl[p].last, gr[r].first,
                                         gr[r].last);
                  if (add3(base, vi, add2(FX(e), gl[p].cost + gr[r].cost)) == v) {
                    emit_edge(D, ex);
                    trace_desc(D, c, l1, &gl[p]);
                    trace_desc(D, b1, l2, &gr[r]);
                    emit_edge(D, eyi);
                    D->tb_energy += e;
                    trace_V(D, c, d, ti);
                    return;
                  }
                }
            }
          }
      }
    /* multiloop */
    if (Ln >= 1 && add3(base, mlclose_fx(&D->P, t), D->D2[IDX(a1, b1)]) == v) {
      emit_edge(D, ex);
      emit_edge(D, eyi);
      D->tb_energy += D->P.mlclosing + D->P.mlintern + D->P.au[t];
      trace_D2(D, a1, b1);
      return;
    }
  }
  tb_fail = 1;
}

static void trace_B(orc_design *D, int a, int b) {
  int N = D->L.N;
  int64_t v = D->Bv[IDX(a, b)];
  for (int t = 0; t < 6; t++)
    if (add2(D->V[IDX(a, b) * 6 + t], beta_fx(&D->P, t)) == v) {
      D->tb_energy += D->P.mlintern + D->P.au[t];
      trace_V(D, a, b, t);
      return;
    }
  tb_fail = 1;
}

/* D2(a,b): edge-extension (in-edge order) before candidate splits in
 * ascending (layer, state id) of the split state c. */
static void trace_D2(orc_design *D, int a, int b) {
  const OLattice *L = &D->L;
  int N = L->N;
  for (;;) {
    int64_t v = D->D2[IDX(a, b)];
    if (v >= ORC_INF) { tb_fail = 1; return; }
    int done = 0;
    for (int k = L->in_off[b]; k < L->in_off[b + 1] && !done; k++) {
      const OEdge *e = &L->edges[L->in_idx[k]];
      if (L->layer[e->from] <= L->layer[a]) continue;
      if (add2(D->D2[IDX(a, e->from)], u_fx(D, e)) == v) {
        emit_edge(D, L->in_idx[k]);
        D->tb_energy += D->P.mlbase;
        b = e->from;
        done = 1;
      }
    }
    if (done) continue;
    for (int c = L->lstart[L->layer[a] + 1]; c < L->lstart[L->layer[b]]; c++) {
      if (!D->cand[IDX(c, b)]) continue;
      if (add2(D->D1[IDX(a, c)], D->Bv[IDX(c, b)]) == v) {
        trace_D1(D, a, c);
        trace_B(D, c, b);
        return;
      }
    }
    tb_fail = 1;
    return;
  }
}

/* D1(a,b): direct branch, left peel (out-edge label order), right peel
 * (in-edge order), then D2. */
static void trace_D1(orc_design *D, int a, int b) {
  const OLattice *L = &D->L;
  int N = L->N;
  for (;;) {
    int64_t v = D->D1[IDX(a, b)];
    if (v >= ORC_INF) { tb_fail = 1; return; }
    if (D->Bv[IDX(a, b)] == v) { trace_B(D, a, b); return; }
    int moved = 0;
    for (int k = L->out_off[a]; k < L->out_off[a + 1] && !moved; k++) {
      const OEdge *e = &L->edges[L->out_idx[k]];
      if (L->layer[e->to] >= L->layer[b]) continue;
      if (add2(u_fx(D, e), D->D1[IDX(e->to, b)]) == v) {
        emit_edge(D, L->out_idx[k]);
        D->tb_energy += D->P.mlbase;
        a = e->to;
        moved = 1;
      }
    }
    if (moved) continue;
    for (int k = L->in_off[b]; k < L->in_off[b + 1]; k++) {
      const OEdge *e = &L->edges[L->in_idx[k]];
      if (L->layer[e->from] <= L->layer[a]) continue;
      if (add2(D->D1[IDX(a, e->from)], u_fx(D, e)) == v) {
        emit_edge(D, L->in_idx[k]);
        D->tb_energy += D->P.mlbase;
        trace_D1(D, a, e->from);
        return;
      }
    }
    if (D->D2[IDX(a, b)] == v) { trace_D2(D, a, b); return; }
    tb_fail = 1;
    return;
  }
}

/* exterior: unpaired out-edges in label order, then branches in ascending
 * (layer of b, state id of b, pair type). */
static void trace_ext(orc_design *D) {
  const OLattice *L = &D->L;
  int N = L->N;
  int a = L->s;
  while (a != L->t && !tb_fail) {
    int64_t v = D->Ext[a];
    int moved = 0;
    for (int k = L->out_off[a]; k < L->out_off[a + 1] && !moved; k++) {
      const OEdge *e = &L->edges[L->out_idx[k]];
      if (add2(e->cost, D->Ext[e->to]) == v) {
        emit_edge(D, L->out_idx[k]);
        a = e->to;
        moved = 1;
      }
    }
    if (moved) continue;
    for (int b = L->lstart[L->layer[a] + 1]; b < N && !moved; b++)
      for (int t = 0; t < 6 && !moved; t++)
        if (add3(D->V[IDX(a, b) * 6 + t], FX(D->P.au[t]), D->Ext[b]) == v) {
          D->tb_energy += D->P.au[t];
          trace_V(D, a, b, t);
          a = b;
          moved = 1;
        }
    if (!moved) tb_fail = 1;
  }
}

static void traceback(orc_design *D, const char *protein, const double *w) {
  int n = D->L.n;
  D->mrna = malloc(n + 1);
  D->structure = malloc(n + 1);
  memset(D->mrna, '?', n);
  memset(D->structure, '.', n);
  D->mrna[n] = D->structure[n] = 0;
  D->tb_energy = 0;
  D->path_cost_fx = 0;
  tb_fail = 0;
  if (D->Ext[D->L.s] >= ORC_INF) tb_fail = 1;
  else trace_ext(D);
  for (int k = 0; k < n; k++) if (D->mrna[k] == '?') tb_fail = 1;
  D->energy = (int32_t)D->tb_energy;
  D->obj_fx = D->Ext[D->L.s];
  if (FX(D->tb_energy) + D->path_cost_fx != D->obj_fx) tb_fail = 1;
  /* FP64 objective re-evaluated from the emitted design, codon order */
  double cc = 0.0;
  if (protein && w && !tb_fail) {
    int A = n / 3;
    for (int k = 0; k < A; k++) {
      int x = -1, y = -1, z = -1;
      for (int c = 0; c < 4; c++) {
        if (D->mrna[3 * k] == NT[c]) x = c;
        if (D->mrna[3 * k + 1] == NT[c]) y = c;
        if (D->mrna[3 * k + 2] == NT[c]) z = c;
      }
      cc += -log(w[16 * x + 4 * y + z]);
    }
  }
  D->codon_cost = cc;
  D->objective = (double)D->energy + (100.0 * D->lambda) * cc;
  D->status = tb_fail ? 1 : 0;
}

/* ------------------------------------------------------------------ */
/* exported API (ctypes)                                                */
/* ------------------------------------------------------------------ */
int orc_run(const char *param_path, const char *protein, const double *w, double lambda,
            orc_design **out) {
  *out = NULL;
  orc_design *D = calloc(1, sizeof(orc_design));
  if (load_params(param_path, &D->P)) { free(D); return -2; }
  if (!(lambda >= 0.0) || !isfinite(lambda)) { free(D); return -1; }
  D->lambda = lambda;
  if (build_codon_lattice(protein, w, lambda, &D->L)) { free(D); return -1; }
  fill(D);
  traceback(D, protein, w);
  *out = D;
  return D->status;
}

/* design under forbidden motifs (comma-separated); returns the traceback
 * status, -1 on invalid input, -3 when no motif-free design exists */
int orc_run_motifs(const char *param_path, const char *protein, const double *w, double lambda,
                   const char *motifs, orc_design **out) {
  *out = NULL;
  orc_design *D = calloc(1, sizeof(orc_design));
  if (load_params(param_path, &D->P)) { free(D); return -2; }
  if (!(lambda >= 0.0) || !isfinite(lambda)) { free(D); return -1; }
  D->lambda = lambda;
  OLattice L0;
  if (build_codon_lattice(protein, w, lambda, &L0)) { free(D); return -1; }
  Matcher *M = malloc(sizeof(Matcher));
  int rc = matcher_build(motifs, M);
  if (rc == 0) rc = motif_product(&L0, M, &D->L);
  free(M);
  lattice_free(&L0);
  if (rc != 0) { free(D); return rc; }
  fill(D);
  traceback(D, protein, w);
  *out = D;
  return D->status;
}

int orc_run_rna(const char *param_path, const char *rna, orc_design **out) {
  *out = NULL;
  orc_design *D = calloc(1, sizeof(orc_design));
  if (load_params(param_path, &D->P)) { free(D); return -2; }
  D->lambda = 0.0;
  if (build_rna_lattice(rna, &D->L)) { free(D); return -1; }
  fill(D);
  traceback(D, NULL, NULL);
  *out = D;
  return D->status;
}

void orc_free(orc_design *D) {
  if (!D) return;
  free(D->H); free(D->V); free(D->Bv); free(D->D1); free(D->D2); free(D->PD);
  free(D->Ext); free(D->cand); free(D->mrna); free(D->structure);
  lattice_free(&D->L);
  free(D);
}

int orc_n(const orc_design *D) { return D->L.n; }
int orc_num_states(const orc_design *D) { return D->L.N; }
int orc_num_edges(const orc_design *D) { return D->L.E; }

void orc_layers(const orc_design *D, int32_t *layer) {
  for (int v = 0; v < D->L.N; v++) layer[v] = D->L.layer[v];
}

/* edges in (from, label) order */
void orc_edges(const orc_design *D, int32_t *from, int32_t *to, int32_t *label, int64_t *cost) {
  for (int k = 0; k < D->L.E; k++) {
    const OEdge *e = &D->L.edges[D->L.out_idx[k]];
    from[k] = e->from; to[k] = e->to; label[k] = e->label; cost[k] = e->cost;
  }
}

/* dense square tables: H, D1, D2, B, PD are N*N; V is N*N*6; Ext is N;
 * cand is N*N bytes (cand[c*N+b]).  Any pointer may be NULL. */
void orc_tables(const orc_design *D, int64_t *H, int64_t *V, int64_t *Bv, int64_t *D1,
                int64_t *D2, int64_t *PD, int64_t *Ext, uint8_t *cand) {
  size_t NN = (size_t)D->L.N * D->L.N;
  if (H) memcpy(H, D->H, NN * 8);
  if (V) memcpy(V, D->V, NN * 48);
  if (Bv) memcpy(Bv, D->Bv, NN * 8);
  if (D1) memcpy(D1, D->D1, NN * 8);
  if (D2) memcpy(D2, D->D2, NN * 8);
  if (PD) memcpy(PD, D->PD, NN * 8);
  if (Ext) memcpy(Ext, D->Ext, (size_t)D->L.N * 8);
  if (cand) memcpy(cand, D->cand, NN);
}

/* result: mrna and structure buffers of n+1 bytes */
void orc_result(const orc_design *D, char *mrna, char *structure, int32_t *energy,
                double *codon_cost, double *objective, int64_t *obj_fx, int64_t *path_cost_fx) {
  if (mrna) memcpy(mrna, D->mrna, D->L.n + 1);
  if (structure) memcpy(structure, D->structure, D->L.n + 1);
  if (energy) *energy = D->energy;
  if (codon_cost) *codon_cost = D->codon_cost;
  if (objective) *objective = D->objective;
  if (obj_fx) *obj_fx = D->obj_fx;
  if (path_cost_fx) *path_cost_fx = D->path_cost_fx;
}

void orc_counts(const orc_design *D, int64_t *Z, int64_t *finite_direct, int64_t *retained) {
  if (Z) *Z = D->Z;
  if (finite_direct) *finite_direct = D->finite_direct;
  if (retained) *retained = D->retained_cells;
}

/* the fixed-point codon cost this oracle uses, exposed for tests */
int64_t orc_codon_cost_fx(double lambda, double w) { return codon_cost_fx(lambda, w); }

/* loop energies exposed for fixture tests (integer dcal/mol) */
int orc_hairpin_energy(const char *param_path, const char *seq) {
  OParams *P = malloc(sizeof(OParams));
  if (load_params(param_path, P)) { free(P); return -999999; }
  int L = (int)strlen(seq) - 2, s[64];
  for (int k = 0; k < L + 2; k++) {
    s[k] = -1;
    for (int c = 0; c < 4; c++) if (seq[k] == NT[c]) s[k] = c;
  }
  int t = pair_type(s[0], s[L + 1]);
  int e = (t < 0 || L < 3) ? -999999 : hairpin_seq_energy(P, t, s, L);
  free(P);
  return e;
}

/* two-loop energy exposed for fixture tests: left = nucleotides i..p (outer
 * 5' end, l1 unpaired, inner 5' end), right = q..j (inner 3' end, l2
 * unpaired, outer 3' end); integer dcal/mol, -999999 on bad input */
int orc_twoloop_energy(const char *param_path, const char *left, const char *right) {
  OParams *P = malloc(sizeof(OParams));
  if (load_params(param_path, P)) { free(P); return -999999; }
  int nl = (int)strlen(left), nr = (int)strlen(right), a[64], b[64];
  if (nl < 2 || nr < 2 || nl > 64 || nr > 64) { free(P); return -999999; }
  for (int k = 0; k < nl; k++) { a[k] = -1; for (int c = 0; c < 4; c++) if (left[k] == NT[c]) a[k] = c; }
  for (int k = 0; k < nr; k++) { b[k] = -1; for (int c = 0; c < 4; c++) if (right[k] == NT[c]) b[k] = c; }
  int l1 = nl - 2, l2 = nr - 2;
  int t = pair_type(a[0], b[nr - 1]), ti = pair_type(a[nl - 1], b[0]);
  int e = (t < 0 || ti < 0 || l1 + l2 > 30)
              ? -999999
              : twoloop_energy(P, t, ti, l1, l2, a[1], a[nl - 2], b[1], b[nr - 2]);
  free(P);
  return e;
}

/* threads used to fill the layer pairs of one span (default 1); returns the
 * previous setting */
int orc_set_threads(int n) {
  int old = g_threads;
  g_threads = n > 0 ? n : 1;
  return old;
}
