/*
 * sd.h -- C ABI of the B300 exact codon-lattice design library (libsd_b300.so).
 *
 * The library computes, for one protein p and weight lambda >= 0 (Sec. 3,
 * Eq. 1 of the SparseDesign paper, arXiv 2609.32308):
 *
 *   F*(p, lambda) = min over synonymous mRNAs r and structures S in S_{3,30}(r)
 *                   of  E_T04,d0(r, S) + lambda * C(r),   C(r) = -sum ln w(c),
 *
 * by the candidate-sparsified span wavefront of Sec. 4.1 / Sec. 5 (Eqs. branch,
 * sparse2, partitionable with S for D, candidates; Algorithm 1) over the
 * layered weighted codon DFA of Sec. 3, on one B300 GPU, followed by a
 * deterministic traceback of the optimal mRNA and structure.
 *
 * Units (Sec. 3): lambda is given in kcal/mol and multiplied by 100 inside;
 * energies are integers in dcal/mol (0.01 kcal/mol).  Internally every DP
 * value is an exact int64 fixed-point number in units of 2^-32 dcal/mol:
 * E * 2^32 + sum over codons of round_half_even(100*lambda * (-ln w) * 2^32).
 * Because this arithmetic is exact, the sparse recurrence equals the dense
 * one bit for bit (Thm. 1) and ties are broken by a fixed canonical order.
 *
 * Threading: an sd_energy is immutable after loading and may be shared by
 * host threads.  A plan is used by one host thread at a time.  All calls are
 * synchronous unless stated; sd_plan_run is asynchronous on the given stream.
 * Errors are returned as negative codes (sd_strerror gives the text); no call
 * aborts the process.
 */
#ifndef SD_B300_H
#define SD_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define SD_OK 0
#define SD_EINVAL (-1)      /* invalid argument (protein, weights, lambda, file)   */
#define SD_ERANGE (-2)      /* objective would leave the exact int64 range         */
#define SD_EINFEASIBLE (-3) /* empty design language (no complete path)            */
#define SD_ENOMEM (-4)      /* host or device allocation failed                    */
#define SD_ECUDA (-5)       /* a CUDA runtime call failed                          */
#define SD_ETIMEOUT (-6)    /* a bounded device wait expired                       */
#define SD_EINTERNAL (-7)   /* traceback could not reproduce the DP value          */
#define SD_ESIZE (-8)       /* design larger than sd_design_noalloc's fixed scratch */

typedef struct sd_energy sd_energy; /* opaque nearest-neighbour parameter set */
typedef struct sd_plan sd_plan;     /* opaque batch of designs resident on the GPU */

/* One design (Sec. 5: the design is checked against its DFA path and a
 * recomputed objective).  Buffers are owned by the result: sd_result_free. */
typedef struct {
  char *mrna;           /* n+1 bytes, A/C/G/U, NUL-terminated                       */
  char *structure;      /* n+1 bytes, dot-bracket, NUL-terminated                   */
  int32_t energy;       /* dcal/mol, dangle-0 free energy of (mrna, structure)      */
  int32_t n;            /* nucleotides = 3 * codon positions                        */
  double codon_cost;    /* C(r) = -sum ln w(c) in FP64, summed in codon order        */
  double objective;     /* energy + (100*lambda) * codon_cost, FP64, dcal/mol        */
  int64_t objective_fx; /* exact DP optimum, units of 2^-32 dcal/mol                */
  int64_t Z;            /* retained candidates, sum_b |C_b| (Eq. candidates)        */
  int64_t finite_direct;/* direct intervals with finite B (B_finite)                 */
  int64_t retained_cells;/* finite V_t, S1, S2 cells + candidate appends            */
  int64_t states, edges;/* DFA size N and |E|                                       */
  int32_t regrows;      /* candidate-buffer regrow passes (0 when presized enough)  */
  int32_t reserved;
} sd_result;

/* Load a nearest-neighbour parameter set (Sec. 3: the Turner-2004 dangle-0
 * model with special hairpins, lonely pairs, minimum hairpin 3 and at most 30
 * unpaired nucleotides per two-loop).
 *   path_or_null    a parameter file in the plain-text "SDENERGY 1" format:
 *                   named integer tables stack[6][6],
 *                   mismatch_{hairpin,interior,interior_1n,interior_23}[6][4][4],
 *                   int11[6][6][4][4], int21[6][6][4][4][4],
 *                   int22[6][6][4][4][4][4], hairpin/bulge/interior[31],
 *                   terminal_au[6], ninio, max_ninio, ml_closing, ml_intern,
 *                   ml_base ("<name> <count>" then the integers, row-major),
 *                   then "lxc <float>" and the special triloop / tetraloop /
 *                   hexaloop lists ("<name> <count>", then "<sequence> <total>"
 *                   lines).  Pair types are AU CG GC UA GU UG; two-loop tables
 *                   are indexed [outer pair][inner pair read from the loop].
 *                   The paper's tables are not shipped (it pins them by digest).
 *   synthetic_seed  used only when path_or_null is NULL: the library then
 *                   generates seeded synthetic integer tables (dcal/mol) with
 *                   Turner-2004 shapes, signs, magnitudes and two-loop rotation
 *                   symmetries (SplitMix64 random numbers; the same seed gives
 *                   the same set on every machine).
 * On success *out owns a host copy and a device copy on the current device;
 * every call that uses it must run with that device current (else
 * SD_EINVAL).  Returns SD_OK, SD_EINVAL (unreadable / malformed file, NULL
 * out), SD_ENOMEM, SD_ECUDA. */
int sd_load_energy(const char *path_or_null, uint64_t synthetic_seed, sd_energy **out);
/* Write the parameter set in the text format above (a set loaded from a seed
 * becomes a file that any reader of the format, or sd_load_energy, loads
 * back).  Returns SD_OK or SD_EINVAL (NULL argument, unwritable path). */
int sd_energy_save(const sd_energy *e, const char *path);
void sd_energy_free(sd_energy *e);

/* Exact design of one protein (Sec. 3, Eq. 1: the minimum over the synonymous
 * mRNAs r of the protein of MFE(r) + 100 lambda C(r), with C(r) the sum over
 * codons of -ln w(codon), and an MFE structure of the minimising r).
 *   protein       one-letter amino acids, optional '*' as the last symbol only
 *                 (an explicit stop adds a codon position; none is implied);
 *                 may be empty; at most 4000 codon positions (12,000 nt).
 *   codon_weights 64 relative adaptiveness values w(c) in (0,1], indexed
 *                 16*x + 4*y + z with A=0 C=1 G=2 U=3; for every amino acid of
 *                 the protein (and '*') the maximum over its codons must be 1.
 *   lambda        >= 0, kcal/mol.
 * Fills *out (caller-owned struct; buffers freed by sd_result_free).
 * Returns SD_OK or SD_EINVAL / SD_ERANGE / SD_ENOMEM / SD_ECUDA / SD_EINTERNAL,
 * SD_EINFEASIBLE when the design language is empty (no complete mRNA; a
 * protein alone always has one, forbidden motifs can remove them all), or
 * SD_ETIMEOUT when a bounded wait inside the fill expired (no design). */
int sd_design(const sd_energy *energy, const char *protein, const double *codon_weights,
              double lambda, sd_result *out);

/* Exact designs of many proteins in one batched launch sequence: Sec. 3, Eq. 1
 * applied to every item independently (one lattice, codon weights and lambda
 * per item; the items share the launches of the span wavefront, Sec. 5).
 *   proteins[count], codon_weights (count*64 values, or 64 if weights_shared),
 *   lambdas[count]; outs[count] and status[count] are caller-owned arrays.
 * One failing item does not stop the others; status[k] holds its code (any
 * code sd_design returns, SD_EINFEASIBLE included).
 * Returns SD_OK if the batch ran (check status[]), else SD_EINVAL (NULL or
 * negative arguments), SD_ENOMEM, SD_ECUDA or SD_EINTERNAL. */
int sd_design_batch(const sd_energy *energy, int count, const char *const *proteins,
                    const double *codon_weights, int weights_shared, const double *lambdas,
                    sd_result *outs, int *status);

void sd_result_free(sd_result *r);
const char *sd_strerror(int code);

/* ---- forbidden motifs (Sec. 3: the codon DFA intersected with a
 *      deterministic forbidden-motif automaton; Sec. 7.3) ---- */

/* Exact designs whose mRNAs contain none of the given motifs.  The codon DFA
 * of each protein is intersected with the Aho-Corasick automaton of the motif
 * set (matcher history crosses codon boundaries; transitions that complete a
 * motif are removed; states that cannot reach the end are trimmed), which
 * keeps the layered path model, so the same exact DP runs on the product.
 *   motifs[nmotifs]  non-empty strings over A C G U of at most 32 nucleotides,
 *                    at most 64 of them (nmotifs = 0: no constraint).
 * Products whose layers hold up to 2 states run on the same kernels as plain
 * designs; wider ones (up to 8 states per layer, at most 32 in-edges per
 * state) on a wide instance of them with forward-packed full tables; wider
 * products give the item SD_ESIZE.  An item with no motif-free design gets
 * SD_EINFEASIBLE.  Otherwise as sd_plan_create / sd_design. */
int sd_plan_create_motifs(const sd_energy *energy, int count, const char *const *proteins,
                          const double *codon_weights, int weights_shared, const double *lambdas,
                          const char *const *motifs, int nmotifs, sd_plan **out,
                          int *item_status);
int sd_design_motifs(const sd_energy *energy, const char *protein, const double *codon_weights,
                     double lambda, const char *const *motifs, int nmotifs, sd_result *out);

/* ---- many values of lambda for one protein (Sec. 10: supported-envelope
 *      and inverse-lambda tools) ---- */

/* Exact designs of one protein at k values of lambda (kcal/mol, >= 0), in one
 * batched launch sequence: outs[k] and status[k] as in sd_design_batch.
 * Returns SD_OK if the batch ran (check status[]), else an error code. */
int sd_design_sweep(const sd_energy *energy, const char *protein, const double *codon_weights,
                    int k, const double *lambdas, sd_result *outs, int *status);

/* The supported lower envelope of F*(p, lambda) = min_r E(r) + 100 lambda C(r)
 * over lam_lo <= lambda <= lam_hi (Eq. 1 is concave and piecewise linear in
 * lambda; each piece is a design optimal on an interval).  lines[] receives
 * the supported designs in order of increasing lambda (non-increasing codon
 * cost), breaks[] (may be NULL) the count-1 lambdas where one line meets the
 * next.  Found by exact designs at the intersections of adjacent lines, all
 * open intersections of a round in one batch.  Lines whose values differ by
 * less than the fixed-point rounding of the DP ((A+1) * 2^-31 dcal/mol) are
 * one line.  lines[] is a caller array of max_lines results (free each with
 * sd_result_free).  Returns SD_OK, SD_ESIZE (more than max_lines lines: the
 * lines found so far are returned, *count <= max_lines, breaks between lines
 * not yet resolved are left 0), SD_EINVAL, or the error of a design. */
int sd_envelope(const sd_energy *energy, const char *protein, const double *codon_weights,
                double lam_lo, double lam_hi, int max_lines, sd_result *lines, double *breaks,
                int *count);

/* The smallest lambda in [0, lam_hi] whose exact design has codon cost
 * C(r) <= target_codon_cost (from the supported envelope on [0, lam_hi]),
 * and that design.  Returns SD_OK, SD_EINFEASIBLE (no design of the envelope
 * reaches the target), SD_ESIZE (more than 256 supported lines), SD_EINVAL,
 * or the error of a design.  *out is freed with sd_result_free. */
int sd_inverse_lambda(const sd_energy *energy, const char *protein, const double *codon_weights,
                      double target_codon_cost, double lam_hi, double *lambda_out,
                      sd_result *out);

/* Exact design of one protein that allocates no device memory.
 * The paper has no counterpart: this entry point exists for callers that may
 * not call cudaMalloc (or an allocator built on it, such as torch's) when they
 * ask for a design, e.g. code working inside a device-memory budget fixed in
 * advance.  Same inputs and results as sd_design, except that the caller
 * provides the output strings: out->mrna and out->structure must point to
 * caller buffers of at least 3*strlen(protein)+1 bytes each (do not pass the
 * result to sd_result_free).  The energy set comes from sd_load_energy, which
 * may run earlier, in set-up code that can allocate.
 * Scratch: a 64 MiB static device array held by every GPU that loads the
 * library until the process exits.  Designs whose tables do not fit (beyond a
 * few hundred nucleotides; at most 400 codon positions) return SD_ESIZE.
 * The first call on a device looks up the array's device address on that
 * device (cudaGetSymbolAddress) and must come before any stream capture.
 * All calls share the scratch: calls that overlap on the GPU (two host
 * threads, or work still in flight) race and must be serialised.
 * Runs on the legacy default stream and returns when the design is complete.
 * Returns SD_OK, SD_EINVAL, SD_ERANGE, SD_ESIZE, SD_ECUDA, SD_EINTERNAL,
 * SD_EINFEASIBLE (empty design language, as for sd_design) or SD_ETIMEOUT. */
int sd_design_noalloc(const sd_energy *energy, const char *protein, const double *codon_weights,
                      double lambda, sd_result *out);

/* ---- plan interface: inputs resident in HBM, asynchronous execution ---- */

/* Validate inputs, build every codon DFA on the host, allocate the packed
 * tables and candidate buffers on the current device and upload the lattices.
 * Items that fail validation are recorded in item_status (caller array of
 * count ints, may be NULL) and skipped by sd_plan_run.  Synchronous. */
int sd_plan_create(const sd_energy *energy, int count, const char *const *proteins,
                   const double *codon_weights, int weights_shared, const double *lambdas,
                   sd_plan **out, int *item_status);

/* The same with a chosen layout of the full tables (H, V, B, S1, S2):
 *   SD_LAYOUT_SPAN   0  layer pair (i, i+g) of span g at cell (g-1)(n+1) -
 *                       (g-1)g/2 + i, 4 state-pair slots per cell (the default:
 *                       the cells of one span are contiguous for the wavefront)
 *   SD_LAYOUT_SQUARE 1  state pair (a, b) at a*N + b (Sec. 5: the square arena)
 *   SD_LAYOUT_PACKED 2  forward-packed (Sec. 5): only pairs (a, b) with b on a
 *                       later layer than a, row by row
 * Results do not depend on the layout; memory and speed do (Sec. 8.2 measures
 * packed against square on the CPU).  Anything else is SD_EINVAL. */
#define SD_LAYOUT_SPAN 0
#define SD_LAYOUT_SQUARE 1
#define SD_LAYOUT_PACKED 2
int sd_plan_create_layout(const sd_energy *energy, int count, const char *const *proteins,
                          const double *codon_weights, int weights_shared, const double *lambdas,
                          int layout, sd_plan **out, int *item_status);

/* Run the fill, the exterior pass and the traceback of every valid item on
 * `stream` (a cudaStream_t; NULL means the legacy default stream).
 * Asynchronous: returns after enqueueing.  Re-running recomputes everything. */
int sd_plan_run(sd_plan *plan, void *stream);

/* Record CUDA events around the phases of later sd_plan_run calls (fill,
 * exterior pass, traceback) on the run's stream; sd_plan_phase_times waits
 * for the last timed run and returns the three durations in milliseconds. */
int sd_plan_set_timing(sd_plan *plan, int enable);
int sd_plan_phase_times(const sd_plan *plan, float *ms3);

/* Algorithmic integer work of the fill, per item (ops[count], caller array):
 * runs a counting variant of the fill (synchronously, on the legacy default
 * stream) in which every min-plus term with finite operands adds
 * 2 * (int64 additions + 1) INT32 slots.  Leaves the tables as sd_plan_run
 * does, but without the exterior pass and the traceback. */
int sd_plan_count_ops(sd_plan *plan, int64_t *ops);

/* Threads cooperating on one layer pair in the fill: 8, 16 or 32, or
 * SD_GROUP_BY_SPAN (0): per span, 8 while the span's layer pairs fill the
 * GPU with resident blocks of the group-8 fill, then 16 while they fill it at
 * group 16, then 32 (the late spans, too small for one wave, give every layer
 * pair more threads).  Anything else is SD_EINVAL.  The default is
 * SD_GROUP_BY_SPAN.  Plans of wide layers (motif products) always run groups
 * of 32.  Results do not depend on the group; speed does.
 * sd_plan_autotune runs the plan once per candidate (synchronously, legacy
 * default stream), keeps the fastest and writes the four fill times (ms, in
 * the order SD_GROUP_BY_SPAN, 8, 16, 32; only the first for wide layers) to
 * ms4 (may be NULL). */
#define SD_GROUP_BY_SPAN 0
int sd_plan_set_group(sd_plan *plan, int group);
int sd_plan_get_group(const sd_plan *plan);
int sd_plan_autotune(sd_plan *plan, float *ms4);

/* Capture the whole run (fill, exterior pass, traceback: one launch per span)
 * into a CUDA graph on the next sd_plan_run and replay the graph on later runs
 * (re-captured when the group size or timing changes).  Off by default. */
int sd_plan_set_graph(sd_plan *plan, int enable);

/* Multi-stream schedule (not in the paper; it only orders work): split the
 * plan's designs over k concurrent CUDA streams (1 <= k <= 16), assigned
 * longest-processing-time first by predicted fill work -- each design's layer
 * pairs, plus, when the plan was presized by the retention predictor, its
 * predicted multiloop candidate visits (sd_plan_create_predicted).  Every
 * stream runs the span wavefront of its own designs, so the late spans of one
 * stream, too small to fill the GPU, overlap with the others.  A run forks
 * from the caller's stream and joins back into it, also inside a captured
 * graph.  Results do not depend on k.  With k > 1 sd_plan_phase_times gives
 * (whole run, 0, 0).  k = 1 restores one launch sequence.  Synchronous: waits
 * for the plan's last run.  Returns SD_OK, SD_EINVAL (NULL plan, k out of
 * range) or SD_ECUDA; sd_plan_get_streams returns the current k. */
int sd_plan_set_streams(sd_plan *plan, int k);
int sd_plan_get_streams(const sd_plan *plan);

/* Number of kernel launches one sd_plan_run enqueues. */
int64_t sd_plan_launches(const sd_plan *plan);

/* Synchronise, copy results to the host and re-evaluate the FP64 objective.
 * outs/status: caller arrays of the plan's item count. */
int sd_plan_results(sd_plan *plan, sd_result *outs, int *status);

/* Device bytes held by the plan. */
int64_t sd_plan_device_bytes(const sd_plan *plan);

/* Copy one item's tables to host arrays in the dense square layout used by
 * tests: state ids are numbered layer by layer, inside a layer by codon
 * prefix in ACGU order.  Arrays (any may be NULL):
 *   layer[N] (int32); H[N*N], S1[N*N], S2[N*N], B[N*N] (int64, 2^62 = +inf);
 *   V[N*N*6] (int64); Ext[N] (int64); cand[N*N] (uint8, cand[c*N+b] = 1 iff
 *   c is in C_b).  Query sizes with sd_plan_item_size. Synchronous. */
int sd_plan_item_size(const sd_plan *plan, int item, int32_t *n, int32_t *N, int32_t *E);
int sd_plan_dump(const sd_plan *plan, int item, int32_t *layer, int64_t *H, int64_t *V,
                 int64_t *B, int64_t *S1, int64_t *S2, int64_t *Ext, uint8_t *cand);
/* Lattice edges of one item in (from, label) order. */
int sd_plan_edges(const sd_plan *plan, int item, int32_t *from, int32_t *to, int32_t *label,
                  int64_t *cost);
void sd_plan_free(sd_plan *plan);

/* ---- retention-count predictor (presizes candidate lists; not in the paper:
 *      the paper retains candidates by the exact test B < P_S of Sec. 4.1,
 *      which stays the only rule deciding what is kept) ---- */

#define SD_PRED_FEATURES 32 /* input channels per codon position */
#define SD_PRED_BANDS 8     /* outputs: span bands 5-7, 8-15, ..., 256-511, >= 512 */
typedef struct sd_predictor sd_predictor;

/* A 1-D convolutional network (4 convolutions of width 5, 32 -> 128 -> 128 ->
 * 128 -> 8 channels, ReLU between) with BF16 weights and FP32 accumulation on
 * the current device.  sd_pred_create draws the weights from a seed. */
int sd_pred_create(uint64_t seed, sd_predictor **out);
void sd_pred_free(sd_predictor *p);
int64_t sd_pred_num_params(void);
/* FP32 master parameters, layer by layer: W[5][cin][cout] then bias[cout]. */
int sd_pred_get_params(const sd_predictor *p, float *params);
int sd_pred_set_params(sd_predictor *p, const float *params);
/* Features of one protein: strlen(protein) * SD_PRED_FEATURES floats (host). */
int sd_pred_features(const char *protein, const double *codon_weights, double lambda,
                     float *feat);
/* Forward pass of B sequences padded to L positions: feats [B][L][32],
 * lengths[B], out [B][L][8] = predicted log1p(counts) (host arrays). */
int sd_pred_forward(sd_predictor *p, int B, int L, const float *feats, const int *lengths,
                    float *out);
/* Mean squared error against targets [B][L][8] over the valid positions and
 * its gradient w.r.t. every parameter (grads may be NULL). */
int sd_pred_gradients(sd_predictor *p, int B, int L, const float *feats, const float *targets,
                      const int *lengths, float *grads, float *loss);
/* One Adam step (beta 0.9 / 0.999) on that loss. */
int sd_pred_train_step(sd_predictor *p, int B, int L, const float *feats, const float *targets,
                       const int *lengths, float lr, float *loss);
/* Training labels from an exact run: counts [A][8] of the retained
 * candidates of one plan item by codon of the right endpoint and span band. */
int sd_plan_retention(const sd_plan *plan, int item, int32_t *counts);

/* A plan whose candidate lists get the room the predictor expects (margin x
 * the predicted count of their codon, plus 8, at most the worst case) instead
 * of the worst case.  Results are identical to sd_plan_create's: a list that
 * outgrows its room is detected on the device, and sd_plan_results then gives
 * the affected designs worst-case room and repeats the run (counted in
 * sd_result.regrows).  Runs the predictor's forward pass (synchronous). */
int sd_plan_create_predicted(const sd_energy *energy, sd_predictor *pred, double margin, int count,
                             const char *const *proteins, const double *codon_weights,
                             int weights_shared, const double *lambdas, sd_plan **out,
                             int *item_status);
/* Scalar-dense control (a switch on the same kernels, for measuring what the
 * sparsification saves): with enable != 0 every finite direct interval B(c,b)
 * enters C_b instead of only those with B < P_S (Eq. candidates).  S1, S2 and
 * every optimum are unchanged (Thm. 1); Z and the work grow, and the canonical
 * split of a tied S2 may differ.  Presized lists that overflow are regrown as
 * usual.  Takes effect on the next sd_plan_run (graphs need no re-capture).
 * NULL plan: SD_EINVAL. */
int sd_plan_set_dense(sd_plan *plan, int enable);

/* Candidate-list entries reserved by a plan (all items), and the entries the
 * same items would reserve with worst-case room (every state at least five
 * layers before the list's end state).  NULL plan: 0. */
int64_t sd_plan_candidate_room(const sd_plan *plan);
int64_t sd_plan_candidate_room_worst(const sd_plan *plan);

/* ---- measurement helper (not in the paper) ---- */

/* Integer add/min throughput of the current device, the roofline
 * denominator of the fill: a kernel with 2048 threads per SM, each running 8
 * independent chains of x = min(x + s, t) in 32-bit (bits = 32) or 64-bit
 * (bits = 64) integers, `iters` x 16 steps per chain, timed with CUDA events
 * (best of three after one warm-up).  *ops_per_s counts the add and the min
 * as one operation each.  Synchronous, legacy default stream; allocates a few
 * MB of device memory.  Returns SD_OK, SD_EINVAL (bits not 32/64, iters <= 0,
 * NULL out) or SD_ECUDA. */
int sd_peak_addmin(int bits, int iters, double *ops_per_s);

#ifdef __cplusplus
}
#endif
#endif /* SD_B300_H */
