/*
 * tn.h -- C ABI of the multiple-amplitude tensor-network contraction library.
 *
 * The library computes exact amplitudes <b|U|0^n> of a quantum circuit for a
 * batch of bitstrings b by contracting the circuit's tensor network along a
 * fixed contraction tree, sliced over a set of bond indices, with every
 * intermediate shared by several bitstrings computed once and reused (the
 * multiple-amplitude "store-and-compute" scheme of the paper's main text,
 * Eq. (1), and SM Sec. III).  Per-slice partial amplitudes are summed in
 * complex128 (first-level slicing, SM Sec. IV.B).
 *
 * Conventions shared by every entry point
 *   - Qubit q of a bitstring is column q of a row-major k x n uint8 array
 *     (values 0/1).  As a basis index, qubit 0 is the most significant bit.
 *   - Gate matrices are row-major complex128 (re, im interleaved), row =
 *     output basis state.  A two-qubit gate on (q0, q1) with q0 < q1 uses the
 *     basis |x_q0 x_q1>, matrix index 2*x_q0 + x_q1 (SM Sec. I).
 *   - Fused network (SM Sec. II): one tensor per two-qubit gate, numbered in
 *     gate order; single-qubit gates and the |0> inputs are absorbed into the
 *     next two-qubit gate on their qubit, the final single-qubit layer into
 *     the last one.  Bond edge e is the wire segment of one qubit between two
 *     consecutive two-qubit gates, numbered in creation order while walking
 *     the two-qubit gates in order and, for each gate (a, b), q in (a, b).
 *     Every qubit must take part in at least one two-qubit gate.
 *   - Contraction tree: SSA pair list of (T-1) x 2 int32, leaves 0..T-1,
 *     pair i creates node T+i, the root is node 2T-2.
 *   - Slicing: sliced_edges[j] takes the value (s >> j) & 1 in slice s,
 *     s in [0, 2^n_sliced).  The amplitude is the sum over all slices.
 *   - Amplitude buffers are complex128 (2 doubles per bitstring), one entry
 *     per *input* row of the bitstring array, duplicates included.
 *
 * Errors: every int-returning call returns TN_OK (0) or a negative code;
 * tn_last_error() then holds a thread-local message.  Nothing is written to
 * caller buffers on a host-side validation error.
 *
 * Ownership: inputs are copied at plan time.  Device memory (workspace and
 * amplitude buffers) belongs to the caller; the library allocates no device
 * memory of its own.  Streams belong to the caller.
 */
#ifndef TN_H
#define TN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    TN_OK = 0,
    TN_EINVAL = -1,       /* malformed circuit, tree, bitstrings or sliced edge */
    TN_ENOMEM = -2,       /* workspace smaller than tn_plan_info.workspace_bytes */
    TN_ECUDA = -3,        /* a CUDA runtime call failed (message has the name) */
    TN_ETIMEOUT = -4,     /* a bounded device-side wait gave up */
    TN_EUNSUPPORTED = -5, /* e.g. an intermediate rank above 40 */
    TN_ESTATE = -6        /* call made in the wrong order (e.g. no workspace) */
};

/* Arithmetic of the pairwise contractions (accumulation is always FP32;
 * the cross-slice sum and XEB are FP64). */
enum {
    TN_FP32 = 0,    /* complex64 operands, FP32 FMA on the CUDA cores */
    TN_TF32 = 1,    /* tensor cores, TF32 operands, FP32 accumulate */
    TN_BF16X3 = 2   /* tensor cores, hi/lo BF16 split, three products */
};

typedef struct {
    int32_t q0, q1;   /* q1 = -1 for a single-qubit gate; q0 < q1 otherwise */
    int32_t layer;    /* informational */
    int32_t pad;
    double m[32];     /* 2x2 (first 8 doubles) or 4x4 complex128, row-major */
} tn_gate;

typedef struct {
    int32_t n_qubits;
    int32_t n_gates;
    const tn_gate *gates;   /* in time order */
} tn_circuit;

typedef struct {
    int64_t workspace_limit;  /* bytes the plan may use; <= 0: 64 GiB */
    int32_t slice_batch_log2; /* sliced edges run side by side in one pass;
                                 -1: largest that fits workspace_limit */
    int32_t rescale;          /* 1: per-instance power-of-two rescaling */
    int32_t fuse;             /* 1: non-branching chains of steps with small
                                 side operands run as one kernel each, their
                                 intermediates never stored (SM Sec. V.C) */
    int32_t fuse_max_bits;    /* d^t: a fused chain's tile holds at most
                                 2^d^t complex entries (SM Sec. V.C);
                                 0: default 7 */
    int32_t graphs;           /* 1: tn_contract captures its launch sequence in
                                 a CUDA graph on first use of a (precision,
                                 batch range, output buffer) and replays it */
    int32_t pad0;
    int64_t open_mask;        /* correlated batches: bit q set leaves output
                                 qubit q open (at most TN_MAX_OPEN); each input
                                 bitstring then stands for its 2^|open|
                                 completions (its values at open qubits are
                                 ignored), see tn_contract */
    int32_t reserved[6];
} tn_options;

#define TN_MAX_OPEN 16

typedef struct {
    int32_t n_tensors, n_edges, n_nodes, n_steps;
    int32_t n_unique;             /* distinct bitstrings */
    int32_t n_sliced, slice_batch_log2, n_batches;
    int32_t max_rank;             /* largest per-instance intermediate rank */
    int32_t n_static_steps;       /* steps independent of the sliced edges */
    double flops_ma;              /* Eq. (1) summed over all slices: 8 per complex MAC */
    double flops_sa;              /* single-amplitude cost of all slices times k_unique */
    double flops_exec;            /* flops the executed schedule performs */
    double bytes_min;             /* algorithmic bytes: every materialised
                                     intermediate written once, read once per use */
    int64_t workspace_bytes;      /* device bytes tn_plan_bind needs */
    int64_t peak_tensor_bytes;    /* largest intermediate set (all instances) */
    int64_t upload_bytes;         /* host-to-device bytes tn_plan_bind copies */
    int64_t launches_per_call;    /* kernels one full tn_contract launches */
    int32_t n_open;               /* open output qubits (tn_options.open_mask) */
    int32_t n_chains;             /* fused chains (tn_options.fuse) */
    int64_t amps_per_row;         /* 2^n_open complex amplitudes per input row */
} tn_plan_info;

typedef struct tn_plan_s *tn_plan_t;

/* Zero-initialised defaults. */
void tn_options_default(tn_options *opt);

/* Structure of the fused network (SM Sec. II).  Host only.
 * edge_ends (2*n_edges int32, earlier tensor first) and out_tensor (n_qubits
 * int32, the tensor carrying each output leg) may be NULL. */
int tn_network(const tn_circuit *circ, int32_t *n_tensors, int32_t *n_edges,
               int32_t *edge_ends, int32_t *out_tensor);

/* Build a plan: fused network, slicing, the static reuse-instance DAG
 * (SM Sec. III), step schedule and workspace layout.  Host only; touches no
 * GPU.  bits: k x n_qubits uint8.  tree_ssa: (T-1) x 2 int32.
 * sliced_edges: n_sliced distinct bond edges (may be NULL if n_sliced = 0). */
int tn_plan(const tn_circuit *circ, const uint8_t *bits, int64_t k,
            const int32_t *tree_ssa, const int32_t *sliced_edges, int32_t n_sliced,
            const tn_options *opt, tn_plan_t *out);

/* Sizes and costs of a plan (host only): the multiple-amplitude cost S_k of
 * Eq. (1) summed over the slices (flops_ma) beside the single-amplitude cost
 * times the distinct bitstrings (flops_sa, the main text's comparison of
 * S_k with k S), the largest per-instance rank, the algorithmic bytes, the
 * workspace tn_plan_bind needs and the batch partition of the slices
 * (SM Sec. IV.B).  TN_EINVAL for null arguments. */
int tn_plan_query(tn_plan_t plan, tn_plan_info *info);

/* Per-node reuse widths w_v (distinct projections of the bitstrings onto
 * the node's output qubits) and per-instance ranks, 2T-1 entries each; the
 * data behind Eq. (1).  Either pointer may be NULL. */
int tn_plan_widths(tn_plan_t plan, int64_t *width_out, int32_t *rank, int32_t *n_slice_vars);

/* One row per step, in execution order (the features a kernel choice
 * depends on): */
typedef struct {
    int32_t node, a, b;       /* tree node produced and its operands (a: larger) */
    int32_t mb, kb, nb;       /* free bits of a, contracted bits, free bits of b */
    int32_t rank_a, rank_b;   /* per-instance ranks of the operands */
    int32_t level;            /* slice-loop level (64: once per call) */
    int32_t kernel;           /* 0 per-row SIMT, 1 tiled GEMM */
    int64_t n_inst, n_inst_a, n_inst_b;  /* instances of the output and operands */
    double flops, bytes;      /* per pass: 8 * n_inst * 2^(mb+kb+nb); A + B reads + C write */
    double runs;              /* passes over all slice batches */
    int32_t a_run_m, a_run_k; /* lowest address bits of an A instance that are
                                 consecutive m (resp. k) bits: contiguous runs */
    int32_t b_run_k, b_run_n;
    int64_t n_groups;         /* runs of output instances sharing one A instance */
    int32_t chain;            /* fused chain holding the step (tn_options.fuse), -1: none */
    int32_t chain_last;       /* 1 if the chain runs at this step (its last) */
    int8_t c_pos_m[40];       /* address bit of C holding each m bit, and each n bit */
    int8_t c_pos_n[24];
    int64_t max_group;        /* output instances in the largest group */
    int64_t n_pair_tiles;     /* N = 64: 64-column tiles with every group padded to an even
                                 count (the tensor cores' column-tile pairs), else 0 */
} tn_step_info;

int tn_plan_steps(tn_plan_t plan, tn_step_info *steps, int32_t n);

/* The slices of slice batch `batch` (main text: first-level slicing sums
 * the partial amplitudes of all 2^n_sliced assignments of the sliced bond
 * indices; SM Sec. IV.B).  tn_contract takes batch ranges: batch b holds
 * 2^slice_batch_log2 slices, whose ids s (sliced_edges[j] = (s >> j) & 1)
 * this call writes to slice_ids (host, n >= 2^slice_batch_log2 entries) in
 * the order the batch's pass computes them.  Over b in [0, n_batches) every
 * slice id appears exactly once.  Host only.  TN_EINVAL for a batch outside
 * [0, n_batches) or too small a buffer. */
int tn_plan_batch_slices(tn_plan_t plan, int64_t batch, int64_t *slice_ids, int64_t n);

/* Bind caller-owned device memory (>= info.workspace_bytes, 256-byte
 * aligned) and upload the plan's tables and gate tensors into it on
 * `stream`.  Must precede tn_contract*. */
int tn_plan_bind(tn_plan_t plan, void *workspace, size_t bytes, void *stream);

/* The contraction (main text: the amplitudes of all requested bitstrings
 * with every shared intermediate computed once, Eq. (1); SM Sec. IV.B: the
 * amplitude is the sum over the slices of the sliced indices' partial
 * amplitudes).  Accumulate into amps (device, complex128, k x amps_per_row
 * entries) the partial amplitudes of every slice in slice batches
 * [batch_lo, batch_hi).
 * With open qubits q_0 < ... < q_{r-1} (tn_options.open_mask), entry
 * p * 2^r + x of input row p is the amplitude of its bitstring with qubit
 * q_i set to bit r - 1 - i of x (the lowest open qubit is the most
 * significant, as in the state-vector index); r = 0: one entry per row.  The plan
 * partitions the 2^n_sliced slices into tn_plan_info.n_batches batches of
 * 2^slice_batch_log2 slices each (its own order of the sliced edges:
 * batch b holds the slices whose looped sliced edges take the bits of b);
 * [0, n_batches) covers every slice once, and disjoint ranges can run on
 * different devices and be summed.  Within a call, a batch re-runs only the
 * steps whose sliced edges changed since the previous batch.  Partials are
 * added in a fixed order (deterministic).  Asynchronous on `stream`. */
int tn_contract(tn_plan_t plan, int precision, int64_t batch_lo, int64_t batch_hi,
                double *amps, void *stream);

/* Partial amplitudes of individual slices (SM Sec. IV.B: one assignment of
 * the sliced indices each), for comparison with an oracle: slice_ids are
 * external slice numbers s (sliced_edges[j] = (s >> j) & 1);
 * partials (device, complex128) receives ns x k x amps_per_row entries,
 * slice-major, rows and completions as in tn_contract, each already scaled
 * back by its power-of-two exponent. */
int tn_contract_slices(tn_plan_t plan, int precision, const int64_t *slice_ids, int32_t ns,
                       double *partials, void *stream);

/* Linear XEB fidelity F = (2^n / k) * sum_b |amp_b|^2 - 1 of k device
 * complex128 amplitudes (the estimator whose mean matches the density of
 * Eq. (fxeb): E[N p] = 1 + F), reduced in FP64 on the device in a fixed
 * order.  Writes one double to the caller's device word *xeb_dev;
 * asynchronous on `stream`. */
int tn_xeb(const double *amps, int64_t k, int32_t n_qubits, double *xeb_dev, void *stream);

/* Perfect samples from correlated batches (main text on Fig. 3(b): a small
 * batch of correlated amplitudes yields one exact sample; SM Sec. II: the
 * batch leaves some output qubits open).  amps: k x 2^n_open device
 * complex128 amplitudes as tn_contract writes them with n_open open
 * qubits; uniform: k device doubles in [0, 1), the caller's random numbers.
 * picks[p] (device int64) = the smallest completion x whose running sum of
 * |amp(p, x)|^2, in x order, exceeds uniform[p] times the batch's total
 * (2^n_open - 1 if none does): x is drawn with probability
 * |amp(p, x)|^2 / sum_x' |amp(p, x')|^2.  FP64 with correctly rounded
 * operations (no fused multiply-add), so the choice is reproducible on a
 * host.  TN_EINVAL for n_open outside [0, TN_MAX_OPEN], k <= 0 or null
 * pointers; asynchronous on `stream`. */
int tn_sample_completions(const double *amps, int64_t k, int32_t n_open, const double *uniform, int64_t *picks,
                          void *stream);

/* Porter-Thomas fit of the fidelity (analysis over tn_xeb's input).  With
 * x_b = 2^n |amp_b|^2, bitstrings drawn from a depolarised ideal output
 * distribution have the density p(x) = e^-x (1 + F (x - 1)) (Eq. (fxeb):
 * the mixture of F x e^-x and (1 - F) e^-x).  tn_pt_moments writes five
 * FP64 sums over the k device complex128 amplitudes to the caller's device
 * words out_dev[0..4]: sum g, sum g^2 with g = (x - 1) / (1 + F (x - 1))
 * (the derivative of the log-likelihood in F and minus its second
 * derivative, the Fisher information), sum log(1 + F (x - 1)), sum x and
 * sum x^2 (the linear XEB F = mean(x) - 1 and its standard error).  One
 * block, fixed summation order.  TN_EINVAL for F outside [0, 1), k <= 0 or
 * null pointers; asynchronous on `stream`. */
int tn_pt_moments(const double *amps, int64_t k, int32_t n_qubits, double fidelity, double *out_dev,
                  void *stream);

/* Histogram of x_b = 2^n |amp_b|^2: counts_dev[j] (device, uint64, nbins + 1
 * words, caller-zeroed, accumulated into) gains the b with
 * floor(x_b / (x_max / nbins)) = j for j < nbins, and counts_dev[nbins]
 * those with x_b >= x_max.  x_b, the bin width and the division are
 * correctly rounded FP64 operations (no fused multiply-add), so a host
 * computing re*re + im*im, times 2^n, divided by x_max / nbins, floored,
 * gets the same bins.  TN_EINVAL for nbins outside [1, TN_PT_MAX_BINS],
 * x_max <= 0, k <= 0 or null pointers. */
#define TN_PT_MAX_BINS 8192
int tn_pt_histogram(const double *amps, int64_t k, int32_t n_qubits, double x_max, int32_t nbins,
                    uint64_t *counts_dev, void *stream);

/* Override the kernel family of one step (-1: the plan's choice; 0: per-row
 * kernel, valid when N <= 16 and K*N <= 256; 1: grouped GEMM -- tensor
 * cores for TN_TF32 / TN_BF16X3 when the shape allows, CUDA cores
 * otherwise), with the first schedule of that family (configuration 0 or
 * 2 below).  TN_EINVAL for a family the step's shape does not allow. */
int tn_plan_set_kernel(tn_plan_t plan, int32_t step, int32_t kernel);

/* ---------------------------------------------------------------------
 * Per-step kernel configuration (config selection; no counterpart in the
 * paper, whose Sunway kernels are fixed): the autotuner measures, and the
 * cost model predicts, each step's time under each configuration.
 *
 * A configuration c in [0, TN_NCONFIG) is a kernel family and a schedule:
 *   0  per-row kernel, blocks of up to 16 row passes   (needs N <= 16, K*N <= 256)
 *   1  per-row kernel, blocks of up to 4 row passes; where M is small,
 *      one output instance row per lane group       (same condition)
 *   2  grouped GEMM, consecutive blocks walk the rows of one column tile
 *      (SIMT) / the column tiles of one row tile (tensor cores)
 *   3  grouped GEMM, the other walk order
 * The GEMM runs on the tensor cores for TN_TF32 / TN_BF16X3 where the shape
 * allows (K >= 8, 64 <= M < 2^31), on the CUDA cores otherwise. */
#define TN_NCONFIG 4

/* Set step `step` to configuration `config` (-1: the plan's own choice).
 * TN_EINVAL for a configuration the step's shape does not allow. */
int tn_plan_set_config(tn_plan_t plan, int32_t step, int32_t config);

/* Tensor-core form of the grouped GEMM.  enable = 1 (the default): where B
 * fits in shared memory (configuration 2: a group's whole B, configuration
 * 3: one 64-column tile's, at most 8 K chunks of 16), each CTA takes a
 * contiguous range of tiles and keeps B resident, streaming only A;
 * elsewhere, and for every step with enable = 0, B is gathered chunk by
 * chunk next to A.  Both forms compute the same values; the switch exists
 * to measure and test the streaming form.  TN_EINVAL for a null plan. */
int tn_plan_set_tc_resident_b(tn_plan_t plan, int32_t enable);

/* Column-tile pairs in the tensor-core BF16x3 form with packed B
 * (configuration 2, N >= 64 per instance, K >= 256): enable = 1 (the default) walks
 * a row tile's column tiles two at a time, one MMA of N = 256 writing both
 * accumulators, so one issued instruction does twice the work (N = 64: two
 * instances of a group; a group of odd size ends with a pad tile whose
 * columns are not stored); 0 walks them one at a time.  Both compute the same values; the switch exists to
 * measure and test the single-tile form.  TN_EINVAL for a null plan. */
int tn_plan_set_tc_pairs(tn_plan_t plan, int32_t enable);

/* Fused chains (tn_options.fuse; SM Sec. V.C fuses a run of steps so that
 * only its last output leaves fast memory).  A chain runs fused (enable = 1,
 * the default: one kernel, intermediates never stored) or as its separate
 * steps (0: each step with its own configuration, its intermediate written
 * to the slot the plan keeps for it); both give the same values up to
 * rounding.  tn_plan_autotune decides per chain by timing both.  TN_EINVAL
 * for a chain outside [0, n_chains). */
int tn_plan_set_chain(tn_plan_t plan, int32_t chain, int32_t enable);
/* Whether each chain runs fused (n entries, 1 or 0). */
int tn_plan_get_chains(tn_plan_t plan, int32_t *enabled, int32_t n);

/* Configuration each step will run with (the plan's choice where none was
 * set); n entries. */
int tn_plan_get_configs(tn_plan_t plan, int32_t *config, int32_t n);

/* Cost-model features: TN_NFEAT floats per step for configuration `config`
 * at `precision` (row-major n_steps x TN_NFEAT, host memory), and whether
 * the configuration is allowed (eligible, n_steps int32, may be NULL).
 * Host only.  Features, all O(1): the operand and output bit counts
 * (mb, kb, nb, ranks), log2 of the instance, group and column counts, the
 * contiguous address runs of A, B and C (the permutation class), log2 of
 * flops and bytes per pass, one-hot precision, kernel family, schedule, and
 * log2 of the output rows. */
#define TN_NFEAT 24
int tn_plan_features(tn_plan_t plan, int precision, int32_t config, float *feat, int32_t *eligible, int32_t n);

/* Exhaustive autotuner.  For every configuration c, run the first slice
 * batch of the contraction (in which every step runs exactly once; `reps` +
 * 1 times, the first discarded) with every selected step (step_mask[s] !=
 * 0, or all steps if step_mask is NULL) that allows c set to c, the others
 * unchanged, and time every step with CUDA events.  times (host, n_steps x TN_NCONFIG, may be NULL)
 * receives the fastest time per pass of each (step, configuration) in ms,
 * NaN where not measured.  Afterwards every selected step is set to its
 * fastest configuration.  amps_scratch: device complex128 buffer of k
 * entries the runs accumulate into (its contents are meaningless
 * afterwards).  Fused chains: the configurations are timed with every
 * chain run as separate steps; then each chain is timed fused and kept
 * fused only where that beats the sum of its steps' best times
 * (tn_plan_set_chain).  Needs a bound workspace; synchronises `stream`. */
int tn_plan_autotune(tn_plan_t plan, int precision, int32_t reps, const uint8_t *step_mask, double *amps_scratch,
                     double *times, void *stream);

/* Cost-model selection: predict log2(ms per pass) of every (step, allowed
 * configuration) with the FP16 network params16 (device, TN_MLP_NPARAMS
 * halves, see tn_mlp_to_half), set each step to its predicted fastest
 * configuration, and flag in uncertain (host, n_steps int32, may be NULL)
 * the steps whose two best predictions lie within `margin` (log2 units):
 * those are the steps to hand to tn_plan_autotune (its step_mask) as the
 * fallback.  scratch: device buffer of at least
 * n_steps * TN_NCONFIG * (TN_NFEAT + 1) * 4 bytes.  Synchronises `stream`. */
int tn_plan_select(tn_plan_t plan, int precision, const uint16_t *params16, float margin, void *scratch,
                   size_t scratch_bytes, int32_t *uncertain, void *stream);

/* ---------------------------------------------------------------------
 * Cost-model network: MLP, TN_MLP_IN inputs, two ReLU hidden layers of
 * TN_MLP_HIDDEN units, one output.  Parameters: one flat FP32 device array
 * of TN_MLP_NPARAMS floats, in order W1 [H][D] (row j = hidden unit j), b1
 * [H], W2 [H][H], b2 [H], w3 [H], b3 [1].  X: device, n x TN_MLP_IN FP32,
 * row-major.  All calls are asynchronous on `stream` and allocate nothing. */
#define TN_MLP_IN TN_NFEAT
#define TN_MLP_HIDDEN 128
#define TN_MLP_NPARAMS (TN_MLP_HIDDEN * TN_MLP_IN + TN_MLP_HIDDEN + TN_MLP_HIDDEN * TN_MLP_HIDDEN + 2 * TN_MLP_HIDDEN + 1)

/* y[i] = network(X[i]) in FP32. */
int tn_mlp_forward(const float *params, const float *X, int64_t n, float *y, void *stream);
/* Gradient of L = (1/n) sum_i (y_i - t_i)^2 with respect to the parameters
 * (grad: device, TN_MLP_NPARAMS floats) and L itself (loss: device float,
 * may be NULL); deterministic (per-block partials summed in a fixed order
 * in `scratch`, device, >= tn_mlp_grad_scratch_bytes(n) bytes). */
size_t tn_mlp_grad_scratch_bytes(int64_t n);
int tn_mlp_grad(const float *params, const float *X, const float *t, int64_t n, float *grad, float *loss,
                void *scratch, size_t scratch_bytes, void *stream);
/* One Adam step (bias-corrected first and second moments m, v: device,
 * TN_MLP_NPARAMS floats each, zero before step 1; step counts from 1). */
int tn_mlp_adam(float *params, const float *grad, float *m, float *v, int32_t step, float lr, float beta1,
                float beta2, float eps, void *stream);
/* FP16 copy of the parameters (round to nearest) for inference. */
int tn_mlp_to_half(const float *params, uint16_t *params16, void *stream);
/* y[i] = network(X[i]) with FP16 weights and activations (FP32 sums every
 * 16 products). */
int tn_mlp_forward_f16(const uint16_t *params16, const float *X, int64_t n, float *y, void *stream);

/* Synchronise `stream` and report device-side failures of earlier calls on
 * this plan: TN_ETIMEOUT if a bounded wait inside a kernel gave up (the
 * flag is then cleared), TN_OK otherwise. */
int tn_plan_check(tn_plan_t plan, void *stream);

/* Device time of each step summed over the slice batches of the last
 * tn_contract* call, when profiling is on (tn_plan_profile(plan, 1): CUDA
 * events around every launch, read back by tn_plan_step_times, which
 * synchronises the events); ms has n_steps entries.  kernel (may be NULL)
 * receives the kernel family each step last ran: 0 per-row SIMT, 1 tiled
 * SIMT GEMM, 2 tensor-core GEMM, 3 fused chain (the chain's time is booked
 * on its last step). */
int tn_plan_profile(tn_plan_t plan, int enable);
int tn_plan_step_times(tn_plan_t plan, double *ms, int32_t *kernel, int32_t n);

/* FP32 fused multiply-add throughput probe (no counterpart in the paper: it
 * measures the denominator of the FP32 form's roofline, the rate of the
 * CUDA cores' FP32 FMA pipes on this device).  Launches `blocks` blocks of
 * 256 threads; every thread performs 16 * iters FP32 flops (8 independent
 * FMA chains), so one launch performs blocks * 256 * 16 * iters flops; the
 * caller times it with events on `stream`.  out_dev: device, >= blocks
 * floats, written only in a case the probe's values never reach (it keeps
 * the work from being optimised away).  TN_EINVAL for blocks outside
 * (0, 2^31), iters < 0 or a null buffer; asynchronous. */
int tn_fma_probe(int64_t blocks, int64_t iters, float *out_dev, void *stream);

/* Contraction for callers that cannot allocate device memory.  No
 * counterpart in the paper.  Some callers cannot call cudaMalloc or take
 * device memory from an allocator: code embedded in a host application
 * whose memory pools are owned by another runtime, or a process whose
 * device memory is fixed before it starts.  For them this entry point runs
 * the same contraction as tn_plan_bind + tn_contract over every slice batch,
 * with the workspace in a fixed device array inside the library
 * (TN_STATIC_SCRATCH_BYTES, 64 MiB, reserved on every device that loads the
 * library until the process exits).  It calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *   amps: caller-owned device complex128 buffer of k x amps_per_row
 *         entries (tn_plan_info; amps_per_row = 2^|open qubits|, 1 without
 *         tn_options.open_mask), accumulated into as in tn_contract.
 *   Plans whose tn_plan_info.workspace_bytes exceed TN_STATIC_SCRATCH_BYTES
 *   are rejected with TN_ENOMEM and a message giving both sizes.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  Every call uploads the plan's tables into the array and clears
 * what must start at zero, because the array keeps the last call's
 * contents; calls that overlap on the GPU (other streams, other threads)
 * share the array and race.  A plan's own tn_plan_bind binding, and the CUDA
 * graphs tn_contract captured for it, are left as they were. */
#define TN_STATIC_SCRATCH_BYTES (64ll << 20)
int tn_contract_static(tn_plan_t plan, int precision, double *amps, void *stream);

void tn_destroy(tn_plan_t plan);

/* Thread-local message of the last failing call ("" if none). */
const char *tn_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TN_H */
