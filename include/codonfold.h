/*
 * codonfold.h -- C ABI of the B300 codon-constrained partition-function library.
 *
 * The library computes, for a protein psi, the partition function summed over
 * every codon sequence that encodes psi and every pseudoknot-free secondary
 * structure of that sequence, under a nearest-neighbour energy model with
 * soft per-codon and per-codon-pair weights; then pair probabilities, codon
 * marginals and exact samples.  Citations are to arXiv 2604.19718
 * (Fornace, Wang & Lindsey).
 *
 * Conventions for every entry point:
 *   - every call returns a cf_status; no C++ exception crosses the ABI;
 *   - output buffers are owned and allocated by the caller; a pointer may be
 *     host memory or device memory of the problem's device (the library asks
 *     the CUDA runtime which it is and copies accordingly); device memory of
 *     another device is rejected with CF_EINVAL wherever a kernel would read
 *     or write the buffer in place (cf_sample, cf_sample_noalloc,
 *     cf_window_logz, the surrogate's window inputs);
 *   - one cf_problem is bound to one device and one CUDA stream; calls on one
 *     problem must not overlap (not thread-safe per problem), distinct
 *     problems are independent;
 *   - on failure, cf_last_error() gives a one-line message for that problem.
 *
 * Amino acids are the 20 standard ones, letters "ARNDCQEGHILKMFPSTWYV".
 * Codon states of a residue are its sense codons in lexicographic order over
 * A,C,G,U ("slot" 0..5).  Sense codon ids 0..60 number the 61 sense codons
 * in the same lexicographic order (stop codons removed).
 */
#ifndef CODONFOLD_H
#define CODONFOLD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cf_model cf_model;
typedef struct cf_problem cf_problem;

typedef enum {
  CF_OK = 0,
  CF_EINVAL = 1,   /* invalid argument (bad letter, size, non-finite weight, NULL) */
  CF_ENOMEM = 2,   /* host or device allocation failed */
  CF_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
  CF_ETIMEOUT = 4, /* a device-side bounded wait gave up; the context stays usable */
  CF_ESTATE = 5,   /* call out of order (e.g. outside before inside) */
  CF_ENUMERIC = 6  /* non-finite or zero partition function after scaling */
} cf_status;

typedef enum {
  CF_FP64 = 0,        /* tables in binary64 with per-diagonal power-of-two exponents */
  CF_FP32_SCALED = 1  /* tables in binary32 with per-diagonal power-of-two exponents;
                         log Z and all normalisations in binary64 */
} cf_precision;

#define CF_NPARAMS 181

/*
 * Load the nearest-neighbour energy model (paper Section "Secondary structure
 * free energy models"; the synthetic parameter layout below).
 *   params:  CF_NPARAMS doubles, energies in kcal/mol:
 *            [0,36) stack[6][6] by pair types AU,CG,GC,UA,GU,UG (outer, inner);
 *            [36,67) hairpin H[L]; [67,98) bulge Bu[L]; [98,129) interior In[L],
 *            L = 0..30; [129,145) terminal mismatch tm[4][4];
 *            [145,161) 5' dangle d5[paired][dangling]; [161,177) 3' dangle d3;
 *            [177] multiloop a, [178] b (per unpaired), [179] c (per branch);
 *            [180] temperature in Celsius.  Bases A,C,G,U = 0..3.
 *   The library copies the values; the caller keeps ownership of params.
 * Errors: CF_EINVAL if params or out is NULL, nparams != CF_NPARAMS or a value
 * is non-finite; CF_ENOMEM.
 */
cf_status cf_load_model(const double *params, size_t nparams, cf_model **out);
cf_status cf_model_free(cf_model *model);

/*
 * Create a problem on CUDA device `device`, issuing all work on `stream`
 * (a cudaStream_t, NULL = the legacy default stream).  The problem keeps a
 * pointer to `model`, which must outlive it.
 * Errors: CF_EINVAL, CF_ECUDA (device cannot be selected), CF_ENOMEM.
 */
cf_status cf_problem_create(const cf_model *model, int device, void *stream, cf_problem **out);
cf_status cf_problem_free(cf_problem *prob);

/*
 * Set the protein and its soft constraints (paper Section "Formulating codon
 * constraints using tensor trains", Eq. pair-tt, and Section "Incorporating
 * soft constraints"): the codon-pair tensor train along the backbone.
 *   aa:         m letters (not NUL-terminated needed), host memory.
 *   codon_logw: m*6 doubles, host memory or NULL (= 0).  Row r, slot s is the
 *               log-weight of the residue's s-th codon; slots >= the number of
 *               codons of that amino acid are ignored.  Enters as e^{+w}.
 *   pair_bonus: 61*61 doubles by sense codon id, host or NULL (= 0); the
 *               log-bonus of codon c at residue r followed by c' at r+1.
 * Allocates the device tables for n = 3m (released by cf_problem_free or the
 * next cf_set_protein).  Invalidates earlier inside/outside results.
 * Errors: CF_EINVAL (m < 1, letter not in the alphabet, non-finite weight),
 * CF_ENOMEM (tables do not fit), CF_ECUDA.
 */
cf_status cf_set_protein(cf_problem *prob, const char *aa, int m, const double *codon_logw,
                         const double *pair_bonus);

/*
 * Replace the soft constraints of the current protein (same meaning and layout
 * of codon_logw and pair_bonus as in cf_set_protein; NULL = 0) without
 * releasing its device tables: the transfer blocks T_p, X_p and residue 0's
 * weights are rebuilt and copied over the old ones.  This is the per-step call
 * of gradient-based weight optimisation (paper Section "Incorporating soft
 * constraints"; the weights enter the tensor train of Eq. pair-tt).
 * Synchronises the problem's stream first; invalidates earlier inside/outside
 * results (cf_outside and cf_sample then return CF_ESTATE until cf_inside).
 * Errors: CF_EINVAL (NULL problem, non-finite weight), CF_ESTATE (no protein
 * set), CF_ECUDA.
 */
cf_status cf_set_weights(cf_problem *prob, const double *codon_logw, const double *pair_bonus);

/*
 * Inside pass (paper Section "Free energy computation", Eq. amino-q): fills
 * the dynamic-programming tables over all intervals by anti-diagonal
 * wavefront on the device and returns log Z (natural log, Z summed over
 * codon sequences and structures, soft weights included) in *logZ (host).
 * Errors: CF_ESTATE (no protein), CF_ENUMERIC, CF_ECUDA, CF_ETIMEOUT.
 */
cf_status cf_inside(cf_problem *prob, cf_precision precision, double *logZ);

/*
 * Outside pass: the hand-written adjoint of the inside pass, in the precision
 * of the last cf_inside.  Any output may be NULL.
 *   pair_prob:  n*n floats, row-major; [i][j] = P(i pairs with j) (Eq.
 *               pair-probability), [i][i] = P(i unpaired).
 *   codon_marg: m*6 doubles; [r][s] = P(residue r uses its codon slot s)
 *               = d log Z / d codon_logw[r][s] (Eq. marginal-codon).
 *   base_marg:  n*4 doubles; [i][b] = P(nucleotide i is base b), bases in the
 *               order A, C, G, U: the sum of the codon marginals of residue
 *               i/3 over its codons with base b at position i%3 (Eq.
 *               marginal-base).
 *   pair_grad:  61*61 doubles; d log Z / d pair_bonus[c][c'] = expected count
 *               of the adjacent codon pair (c, c') summed over residues.
 * Each output pointer may be host or device memory (detected per pointer);
 * the library writes it and keeps no reference.
 * Errors: CF_ESTATE (no inside), CF_EINVAL, CF_ECUDA, CF_ETIMEOUT (a bounded
 * device wait for staged inputs gave up; the outputs are then not valid).
 */
cf_status cf_outside(cf_problem *prob, float *pair_prob, double *codon_marg, double *base_marg, double *pair_grad);

/*
 * Draw `nsamples` exact i.i.d. samples of (codon sequence, structure) from
 * the Boltzmann distribution by stochastic traceback of the inside tables
 * (paper Section "Sequence sampling").  Sample k depends only on (seed, k):
 * the same seed gives bit-identical output for any launch shape.
 *   codons:  nsamples*m int32, sense codon id per residue.
 *   partner: nsamples*n int32, pairing partner per position or -1.
 * Errors: CF_ESTATE (no inside), CF_EINVAL (also: an output in device memory
 * of another device), CF_ENOMEM, CF_ECUDA.
 */
cf_status cf_sample(cf_problem *prob, int nsamples, uint64_t seed, int32_t *codons,
                    int32_t *partner);

/*
 * Minimum free energy (paper Section "Minimization", Eq. min-problem): the
 * minimum over codon sequences encoding the protein and structures of
 *   E(sequence, structure) - kT (sum of codon log-weights + sum of codon-pair
 *   bonuses)                                              [kcal/mol],
 * computed by the recursions of cf_inside in the min-sum semiring (SI
 * "Generalization via evaluation algebras"), and one configuration that
 * attains it (traceback).  Uses the protein and weights of the last
 * cf_set_protein / cf_set_weights; needs no cf_inside.
 * Arithmetic is exact: every elementary energy term and every weight term
 * -kT w (kT = 1.98717e-3 (T + 273.15), binary64) is rounded once, half away
 * from zero, to a multiple of 2^-32 kcal/mol, and the recursions add these
 * integers (int64), so the minimum does not depend on evaluation order.
 *   cost:     the minimum as an integer count of 2^-32 kcal/mol (host), or NULL.
 *   mfe_kcal: the same in kcal/mol (host), or NULL.
 *   codons:   m int32 sense codon ids of a minimiser, host or device, or NULL.
 *   partner:  n int32 pairing partners of the minimiser (-1 unpaired), host or
 *             device, or NULL.  With both NULL no traceback runs.
 * Where several configurations attain the minimum, the traceback returns the
 * first in its fixed order of alternatives.  Allocates the pass's integer
 * tables on the first call for a protein length (10 tables of n(n+1)/2 blocks
 * of 36 int64, about 1.2 GB at n = 900).
 * Errors: CF_EINVAL (NULL problem, an output on another device), CF_ESTATE (no
 * protein), CF_ENOMEM, CF_ECUDA, CF_ENUMERIC (traceback inconsistency).
 */
cf_status cf_mfe(cf_problem *prob, int64_t *cost, double *mfe_kcal, int32_t *codons, int32_t *partner);

/* Device time in milliseconds of the last cf_mfe (pass and traceback). */
float cf_mfe_last_ms(const cf_problem *prob);

/*
 * Suboptimal configurations (paper SI "Suboptimal sequence generation", Alg.
 * subopt, over the min-sum recursions of cf_mfe): every (codon sequence,
 * structure) of the current protein whose integer cost is at most the
 * minimum plus floor(gap_kcal * 2^32) (the 2^-32 kcal/mol grid of cf_mfe),
 * each exactly once, in depth-first order of the recursions.  Up to max_out
 * of them are written to host arrays: cost[max_out] (may be NULL), codons
 * [max_out][m] sense codon ids (may be NULL), partner [max_out][n] (-1
 * unpaired; may be NULL); *count receives the number found, max_out + 1 if
 * there are more (the enumeration stops there).  The MFE tables are
 * computed on the device and one CTA enumerates, for at most 30 s of device
 * time or 5e7 steps (else CF_ENUMERIC; a smaller gap or max_out keeps it
 * short); cf_mfe_last_ms reports the time.  The search keeps the states
 * and partners of the configuration it builds (8 n bytes) and its 512
 * deepest frames in shared memory, hence n <= CF_SUBOPT_MAX_N.  Errors: CF_EINVAL (NULL problem or count,
 * gap < 0 or > 1e6, max_out < 0, device outputs, n > CF_SUBOPT_MAX_N), CF_ESTATE (no protein), CF_ENUMERIC (no finite
 * configuration, an inconsistency), CF_ENOMEM, CF_ECUDA.
 */
#define CF_SUBOPT_MAX_N 20000
cf_status cf_subopt(cf_problem *prob, double gap_kcal, int max_out, int64_t *cost, int32_t *codons,
                    int32_t *partner, int *count);
/* Element expansions (search steps) of the last successful cf_subopt; 0 for
 * a NULL problem or before the first call. */
long long cf_subopt_steps(const cf_problem *prob);

/*
 * Position-state layout (paper Eq. single-tt, Section "Incorporating hard
 * constraints"): 0 (default) codon states, the codon-pair tensor train of
 * Eq. pair-tt (every position of a residue carries the residue's codon);
 * 1 the single-codon tensor train: the first position of a residue carries
 * its distinct first bases, the second its distinct (first, second) base
 * pairs, the third its distinct third bases, and the codon (with its
 * weight lw) is fixed by the transfer from the second position to the
 * third.  Layout 1 has fewer states per position (1.61 against 2.84 on a
 * Dirichlet(1) composition, 1.68 on a uniform one; every position needs at
 * least its number of distinct bases, 1.59 and 1.65) and the same log Z,
 * pair probabilities, codon
 * and base marginals; it has no codon-pair bonuses (cf_set_protein and
 * cf_set_weights reject pair_bonus != NULL, cf_outside a pair_grad output),
 * and every other call serves both layouts: in layout 1 the samplers, the
 * MFE traceback and the suboptimal search read a residue's codon off the
 * states of its second and third positions, and the MFE and its
 * suboptimal sets are the same as with codon states (integer costs).
 * cf_set_layout takes effect at the next cf_set_protein; a batch keeps
 * layout 0.  cf_layout_states reports the current protein's layout and, if
 * states != NULL, its n per-position state counts.
 * Errors: CF_EINVAL (NULL problem, unknown layout, layout 1 on a batch).
 */
cf_status cf_set_layout(cf_problem *prob, int layout);
cf_status cf_layout_states(const cf_problem *prob, int *layout, int *states);

/*
 * The paper's own tensor-based free energy model (SI "Tensor-based free
 * energy models", Eq. general-model) under the codon constraints of the
 * problem's protein: gamma x gamma matrices V_x for an unpaired base x
 * (A, C, G, U = 0..3), B^rho_{x,y} for the two sides of a base pair
 * (rho = 0..nrho-1) and S for the weighted trace Tr_S[X] = tr(S X).  A
 * structure's weight is the sum over one rho per pair of the product over
 * its loops (the exterior loop included) of Tr_S[the loop's matrices in
 * backbone order]: V for an unpaired base, B^rho_{x,y} for a base x whose
 * next base in the loop is its partner y, the identity otherwise; pairs
 * closer than 4 positions have no weight.  Codon sequences weigh as in
 * cf_set_protein / cf_set_weights (Eq. amino-q, codon-pair tensor train).
 *
 * cf_tm_spectral_radius: host only (no device use): the spectral radius of a
 *   dim x dim row-major matrix (1 <= dim <= 64), by Gelfand's formula over 48
 *   repeated squarings.  Errors: CF_EINVAL (NULL, bad dim, non-finite entry).
 * cf_tm_model_create: V = 4 x gamma x gamma, B = nrho x 4 x 4 x gamma x gamma
 *   (B[rho][x][y]: x the base whose next loop base is its partner y), S =
 *   gamma x gamma, all row-major binary64 host arrays, copied; 1 <= gamma
 *   <= 4, 1 <= nrho <= 4.  normalize != 0 applies the spectral-radius
 *   renormalisation of SI "Free energy model renormalization": V_x / r_x and
 *   B^rho_{x,y} / sqrt(r_x r_y), r_x the spectral radius of V_x (reported by
 *   cf_tm_model_radius).  The model lives on `device`.  Errors: CF_EINVAL
 *   (NULL, sizes, non-finite entry, a V_x with radius 0 when normalising),
 *   CF_ENOMEM, CF_ECUDA.
 * cf_tm_inside: log Z (natural log) of the problem's protein under the model
 *   into *logZ (host), by the recursion of Eq. complicated-pf with the fold of
 *   Eq. fold generalised to codon states (Eq. design-fold), evaluated by
 *   interval length on the device; CF_FP32_SCALED keeps per-length
 *   power-of-two exponents, CF_FP64 is plain binary64 with the same
 *   exponents.  Tables of about 3 x n(n+1)/2 x 576 values of the precision
 *   are allocated on the first call for a protein and freed with it.  Errors:
 *   CF_EINVAL (NULL, unknown precision, model on another device, a batch),
 *   CF_ESTATE (no protein), CF_ENUMERIC (non-finite or zero Z), CF_ETIMEOUT
 *   (a bounded wait for staged blocks gave up; the problem stays usable),
 *   CF_ENOMEM, CF_ECUDA.
 * cf_tm_last_ms: device time of the last cf_tm_inside.
 */
typedef struct cf_tm_model cf_tm_model;
cf_status cf_tm_spectral_radius(const double *A, int dim, double *radius);
cf_status cf_tm_model_create(int device, int gamma, int nrho, const double *V, const double *B, const double *S,
                             int normalize, cf_tm_model **out);
cf_status cf_tm_model_radius(const cf_tm_model *model, double *radius4);
cf_status cf_tm_model_free(cf_tm_model *model);
cf_status cf_tm_inside(cf_problem *prob, const cf_tm_model *model, cf_precision precision, double *logZ);
float cf_tm_last_ms(const cf_problem *prob);

/*
 * Checkpointing of the interior-loop partial sums (the adjoint's largest
 * intermediate: 29 blocks per cell, 19 GB in binary32 at 3000 nt when stored
 * whole).  Checkpointed, the inside pass keeps them for two diagonals plus
 * every 64th diagonal, and the outside pass recomputes each block of 64
 * diagonals from its checkpoint just before it needs it (same recursion, same
 * operation order: identical values), so the outside pass needs 2 blocks
 * instead of the whole table; the sampler evaluates them from their
 * definition.  mode: -1 (default) checkpointed from CF_CHECKPOINT_MIN_N bases
 * on, 0 never, 1 always.  Takes effect at the next cf_inside (the tables of
 * the current protein are released).  cf_checkpointed reports the form of the
 * current tables (or the one the next cf_inside will use).
 * Errors: CF_EINVAL (NULL problem, unknown mode), CF_ECUDA.
 */
#define CF_CHECKPOINT_MIN_N 3000
cf_status cf_set_checkpoint(cf_problem *prob, int mode);
int cf_checkpointed(const cf_problem *prob);

/*
 * Batches of small proteins of one length (the throughput form of short
 * proteins: paper Section "Computational details" benchmarks random
 * proteins): nprot proteins of m residues, inside and outside in one launch
 * per kernel for the whole batch instead of one graph per protein.  Each
 * protein's arrays occupy one slab of a single device allocation; results
 * equal those of cf_inside / cf_outside on each protein alone.
 *   cf_batch_create: 1 <= m <= CF_BATCH_MAX_M, nprot >= 1, one precision.
 *     Allocates nprot slabs (about 2.6 MB each at m = 8 in binary32).
 *   cf_batch_set_proteins: aa = nprot * m letters (host), codon_logw =
 *     nprot * m * 6 doubles or NULL (layout of cf_set_protein, protein after
 *     protein), pair_bonus = 61 * 61 doubles shared by all proteins or NULL.
 *   cf_batch_run: logZ = nprot doubles (host); pair_prob = nprot * n * n
 *     floats and codon_marg = nprot * m * 6 doubles (host or device), each
 *     may be NULL.  Layouts per protein as in cf_outside.
 *   cf_batch_last_ms: device time of the last run (inside + outside).
 * Errors: CF_EINVAL, CF_ENOMEM, CF_ECUDA, CF_ESTATE (run before set),
 * CF_ENUMERIC, CF_ETIMEOUT; messages from cf_last_error(NULL).
 */
#define CF_BATCH_MAX_M 16
typedef struct cf_batch cf_batch;
cf_status cf_batch_create(const cf_model *model, int device, void *stream, int nprot, int m, cf_precision precision,
                          cf_batch **out);
cf_status cf_batch_set_proteins(cf_batch *batch, const char *aa, const double *codon_logw, const double *pair_bonus);
cf_status cf_batch_run(cf_batch *batch, double *logZ, float *pair_prob, double *codon_marg);
float cf_batch_last_ms(const cf_batch *batch);
cf_status cf_batch_free(cf_batch *batch);

/* One-line description of the last failure on `prob` (or of the last global
 * failure when prob is NULL).  Valid until the next call on that problem. */
const char *cf_last_error(const cf_problem *prob);

/*
 * Device time of the last inside and outside pass in milliseconds, measured
 * with CUDA events on the problem's stream around the kernel sequence, and
 * the number of kernel launches each issued.  Any pointer may be NULL.
 */
cf_status cf_last_timing(const cf_problem *prob, float *inside_ms, float *outside_ms,
                         int *inside_launches, int *outside_launches);

/* Length n = 3m of the current protein, or 0. */
int cf_problem_length(const cf_problem *prob);

/*
 * Batched partition functions of fixed sequences (one codon per residue, so a
 * single state per position): the structure-only dynamic program of paper
 * Section "Dynamic programs over structures for a given sequence" with the
 * same nearest-neighbour loop energies as cf_inside.  Used to label windows of
 * designed sequences with their ensemble free energy G = -RT ln Z.
 *   bases:   concatenated base codes (A, C, G, U = 0..3), one byte each, host
 *            or device memory; window w is bases[offsets[w] .. offsets[w+1]).
 *   offsets: nwin + 1 int64, host or device, non-decreasing, offsets[0] >= 0;
 *            window lengths 0 .. CF_WINDOW_MAX_N (a window shorter than 5 has
 *            no pair and log Z = 0).
 *   logz:    nwin doubles (host or device): natural log of Z of each window.
 * Runs in FP32 with per-diagonal power-of-two exponents and a double exterior
 * sum, one CTA per window.  Needs only the problem's model, device and stream
 * (no protein); scratch is owned by the problem and reused across calls.
 * Errors: CF_EINVAL (NULL argument, nwin < 0, decreasing offsets, window too
 * long, base code > 3), CF_ENUMERIC, CF_ENOMEM, CF_ECUDA.
 */
#define CF_WINDOW_MAX_N 1024
cf_status cf_window_logz(cf_problem *prob, const uint8_t *bases, const int64_t *offsets, int nwin,
                         double *logz);

/* Device time in milliseconds of the last cf_window_logz kernel. */
float cf_window_last_ms(const cf_problem *prob);

/*
 * Learned window free-energy surrogate (the paper has no counterpart: it
 * scores every candidate exactly).  A 1-D convolutional network predicts the
 * ensemble free energy G (kcal/mol) of a window of bases; it is trained on
 * windows labelled by cf_window_logz (G = -RT ln Z) and used to pre-screen
 * candidate codon choices before the exact DP re-scores the best of them.
 *   h0 = one-hot bases; h_l = relu(b_l + W_l * h_{l-1}), l = 1..4, 64
 *   channels, 5 taps, zero padding; g = mean over positions of wh . h4 + bh;
 *   prediction n g.  Loss (1/B) sum (g - G/n)^2, Adam (0.9, 0.999, 1e-8).
 * Parameters: CF_SURROGATE_NPARAMS floats in the order W1 [64][4][5], b1 [64],
 * W2 [64][64][5], b2, W3, b3, W4, b4, wh [64], bh [1].  Convolution weights
 * are applied as BF16 (rounded from the FP32 masters after every update),
 * accumulation is FP32.  Windows: bases as in cf_window_logz, lengths
 * 0..CF_SURROGATE_MAX_LEN.  All buffers may be host or device memory.  Work
 * is issued on `stream`; each call returns after its results are written.
 * Errors: CF_EINVAL (NULL argument, window too long, batch larger than
 * max_batch in training calls, lr <= 0), CF_ENOMEM, CF_ECUDA; the message is
 * read with cf_last_error(NULL).
 */
#define CF_SURROGATE_NPARAMS 63041
#define CF_SURROGATE_MAX_LEN 256
typedef struct cf_surrogate cf_surrogate;
cf_status cf_surrogate_create(int device, void *stream, int max_batch, cf_surrogate **out);
cf_status cf_surrogate_free(cf_surrogate *sur);
/* Replace the parameters (and reset the optimiser state). */
cf_status cf_surrogate_set_params(cf_surrogate *sur, const float *params);
cf_status cf_surrogate_get_params(const cf_surrogate *sur, float *params);
/* Predicted G of nwin windows (any nwin; processed max_batch at a time on
 * the CUDA cores, up to 65,536 windows at a time on the tensor cores, whose
 * row buffers -- about 5 bytes per base -- grow on first use). */
cf_status cf_surrogate_predict(cf_surrogate *sur, const uint8_t *bases, const int64_t *offsets, int nwin,
                               float *G_out);
/* Loss and its gradient (CF_SURROGATE_NPARAMS floats) on one batch, no update. */
cf_status cf_surrogate_grad(cf_surrogate *sur, const uint8_t *bases, const int64_t *offsets, int nwin,
                            const float *G_target, float *loss_out, float *grad_out);
/* One Adam step with learning rate lr on one batch; loss_out may be NULL. */
cf_status cf_surrogate_train_step(cf_surrogate *sur, const uint8_t *bases, const int64_t *offsets, int nwin,
                                  const float *G_target, float lr, float *loss_out);
/* Device time in milliseconds of the last predict or train step. */
float cf_surrogate_last_ms(const cf_surrogate *sur);

/*
 * Which units run cf_surrogate_predict (training always uses the CUDA-core
 * kernels with FP32 activations):
 *   1 (default) tensor cores: the four layers and the head term of a tile
 *     of 116 rows in one persistent kernel, each 64-channel layer a 5-tap
 *     GEMM of 128 rows on the 5th-generation tensor cores (tcgen05 MMA, FP32
 *     accumulator in tensor memory, weights staged by TMA, activations kept
 *     in shared memory between layers); activations carried as two BF16
 *     parts hi + lo (within 2^-18 relative of FP32);
 *   0 CUDA cores: FP32 activations, FP32 FMA.
 * Errors: CF_EINVAL (NULL surrogate, unknown path).  A bounded wait of the
 * tensor-core pipeline that gives up makes cf_surrogate_predict return
 * CF_ETIMEOUT.
 */
cf_status cf_surrogate_set_path(cf_surrogate *sur, int path);

/*
 * cf_sample_noalloc -- the sampler of cf_sample for callers that cannot
 * allocate device memory.  (The paper has no counterpart: this is a library
 * service, not part of the method.)
 *
 * Who needs it: code that runs under a device-memory budget owned by another
 * allocator (for example a framework's caching allocator that has reserved the
 * device), and latency-critical loops in which cudaMalloc/cudaFree would block
 * or synchronise the device.  This entry point calls no cudaMalloc, cudaFree or
 * allocating library routine: the per-warp traceback stacks, per-position
 * states and the error word live in one static device array of
 * CF_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds until
 * the process exits.
 *
 *   Same arguments and results as cf_sample, except that codons (nsamples*m
 *   int32) and partner (nsamples*n int32) must be device memory of the
 *   problem's device.  The inside tables must exist (cf_inside first); they
 *   were allocated by cf_set_protein / cf_inside, not by this call.
 *   Limits: n = 3m <= CF_NOALLOC_MAX_N; CF_NOALLOC_WARPS warps draw samples.
 *   The array holds an error word (256 bytes), the per-warp position states
 *   (CF_NOALLOC_WARPS * CF_NOALLOC_MAX_N int32) and the per-warp traceback
 *   stacks (CF_NOALLOC_WARPS * (CF_NOALLOC_MAX_N + 64) pairs of int32):
 *   CF_NOALLOC_SCRATCH_BYTES = 4,673,792 bytes at the limits below.
 *   Errors: CF_EINVAL (n above the limit, host or NULL output pointers,
 *   nsamples < 0), CF_ESTATE (no inside), CF_ECUDA, CF_ENUMERIC.
 *   Set-up: the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 *   Sharing: all calls in the process share the one array and it keeps the
 *   last call's contents; the call clears what must start at zero.  Calls
 *   whose kernels overlap on the GPU (other streams, other threads, other
 *   problems on the same device) race on the array and must be serialised by
 *   the caller.
 */
#define CF_NOALLOC_MAX_N 3000
#define CF_NOALLOC_WARPS 128
#define CF_NOALLOC_SCRATCH_BYTES                                                              \
  (256 + ((CF_NOALLOC_WARPS * CF_NOALLOC_MAX_N * 4 + 255) / 256) * 256 +                     \
   CF_NOALLOC_WARPS * (CF_NOALLOC_MAX_N + 64) * 8)
cf_status cf_sample_noalloc(cf_problem *prob, int nsamples, uint64_t seed, int32_t *codons,
                            int32_t *partner);

/*
 * Far-band diagnostics of the last binary32 passes (the paper has no
 * counterpart: this reports how the library summed the bifurcation terms).
 * The split points far from the wavefront are summed in tiles whose
 * power-of-two factors follow a linear fit ("chord") of the per-diagonal
 * exponents; a band whose exponents depart from the chord by more than 48
 * (log2) is not tiled but summed term by term with exact factors.
 *   in_max_dev / out_max_dev: largest departure seen by the inside bands and
 *   by the outside pass; in_untiled: inside bands summed term by term;
 *   out_untiled: 1 if the outside pass gathered every term per diagonal;
 *   spread_bits: the spread (log2) of the strengths of the intervals of one
 *   length (lengths up to 400 nt), estimated after the inside pass from the
 *   exterior prefix; past 120 bits the binary32 inside pass returns
 *   CF_ENUMERIC and asks for
 *   CF_FP64 (a composition that changes strongly along the protein spreads
 *   them beyond what binary32 holds).
 * Any pointer may be NULL.  Synchronises the problem's stream.
 * Errors: CF_EINVAL (NULL problem), CF_ECUDA.
 */
cf_status cf_far_band_info(const cf_problem *prob, int *in_max_dev, int *in_untiled, int *out_max_dev,
                           int *out_untiled, int *spread_bits);

/*
 * Test hooks (the paper has no counterpart).  They exist so that tests can
 * drive the library's failure paths without faulting a GPU.
 *   cf_debug_set_wait_polls: the number of polls after which the bounded
 *     waits for staged inputs give up on `device` (default 2^22, about a
 *     second).  With 0 every such wait gives up at once: the kernel records
 *     the timeout, still waits (bounded) for its own copies in flight, and
 *     returns, and cf_inside / cf_outside report CF_ETIMEOUT.  Synchronises
 *     the device before and after; affects every problem on that device.
 *   cf_debug_set_far_dev_max: the departure bound above which a far band is
 *     summed term by term (default 48); 0 sends every band of every binary32
 *     pass on `device` that way.  Synchronises the device.
 *   cf_debug_set_range_limit: the spread (bits) above which the binary32
 *     inside pass on `device` refuses (default 120), and the longest
 *     interval length the spread is measured over (default 400; 0: all).
 *     Synchronises the device.
 *   cf_debug_fail_alloc: after `after` further successful device allocations
 *     of the library (process-wide), the next one fails as if the device were
 *     out of memory (CF_ENOMEM); negative turns the hook off.  The failing
 *     call leaves the problem usable: a failed cf_set_protein leaves no
 *     protein, a failed cf_inside / cf_outside leaves no tables of that
 *     precision.
 *   cf_debug_classify_pointer: the rule by which caller buffers are accepted,
 *     for a pointer with the given cudaMemoryType and device, seen from a
 *     problem on problem_device: 0 host memory, 1 device memory the problem
 *     may use in place, -1 device memory of another device (rejected).
 */
cf_status cf_debug_set_wait_polls(int device, unsigned long long polls);
cf_status cf_debug_set_far_dev_max(int device, int bound);
cf_status cf_debug_set_range_limit(int device, int bits, int max_length);
cf_status cf_debug_fail_alloc(long long after);
int cf_debug_classify_pointer(int memory_type, int pointer_device, int problem_device);

#ifdef __cplusplus
}
#endif

#endif /* CODONFOLD_H */
