/*
 * iqs.h -- C ABI of the GB300 (sm_103a) state-vector gate engine.
 *
 * Operations follow arXiv 2001.10554 ("Intel Quantum Simulator"): a register
 * holds the 2^n complex amplitudes alpha_i of an n-qubit pure state, with
 * index i = sum_q i_q 2^q, so qubit q is bit q and qubit 0 the least
 * significant bit (Section 2, "Distributed implementation", Eq. 1 and the
 * binary index notation before it).  The whole state lives in the memory of
 * one GPU; there is no sharding and no inter-GPU communication.
 *
 * Memory layout: amplitudes are stored interleaved (re, im), contiguous, in
 * index order -- complex64 = 8 bytes (two float32), complex128 = 16 bytes
 * (two float64) per amplitude.  This is the layout of a 1-D torch.complex64
 * / torch.complex128 CUDA tensor.
 *
 * Arithmetic: complex64 registers compute gates in FP32.  complex128
 * registers compute gates either in native FP64 or, by default on large
 * states, in a double-float emulation on the FP32 pipe (the sm_103a FP64 pipe
 * is far too slow to keep pace with HBM); the emulation keeps about 47
 * significant bits per operation.  Every reduction (norm, probability,
 * expectation, energy) accumulates in at least FP64-equivalent precision for
 * both dtypes.
 *
 * Conventions for every function:
 *   - Matrices U are 2x2 complex, row-major, as 8 doubles
 *     {Re U00, Im U00, Re U01, Im U01, Re U10, Im U10, Re U11, Im U11},
 *     always given in FP64 on the host (rounded to FP32 for complex64).
 *   - Calls are ordered on the register's CUDA stream and asynchronous,
 *     except those that return a host value (they synchronise that stream).
 *   - Host pointers are only read during the call; the caller keeps
 *     ownership of every pointer it passes.
 *   - Every call returns an iqs_status and never aborts or prints.  On
 *     IQS_EINVAL the register's state is left untouched; IQS_ERANGE reports
 *     out-of-range amplitudes met by earlier emulated complex128 kernels;
 *     iqs_last_error() gives a message (thread-local).
 */
#ifndef IQS_H
#define IQS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct iqs_reg iqs_reg; /* opaque register handle */

typedef enum { IQS_C64 = 0, IQS_C128 = 1 } iqs_dtype;

typedef enum {
  IQS_OK = 0,
  IQS_EINVAL = 1,    /* bad argument: qubit out of range, c == t, bad Pauli character, size mismatch */
  IQS_ENOMEM = 2,    /* device or pinned-host allocation failed */
  IQS_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
  IQS_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
  IQS_EINTERNAL = 5, /* internal consistency check failed */
  IQS_ERANGE = 6     /* an amplitude outside the emulated-FP64 range was met (|a| >= 2^64, Inf or NaN) */
} iqs_status;

typedef enum {
  IQS_MATH_AUTO = 0,     /* complex128: native FP64 below 2^20 amplitudes, emulated above */
  IQS_MATH_EMULATED = 1, /* complex128: double-float on the FP32 pipe */
  IQS_MATH_NATIVE = 2    /* complex128: native FP64 (DFMA) */
} iqs_math;

#define IQS_MAX_QUBITS 34

/* ------------------------------------------------------------ registers */

/* Section 2 "Scope and basic use": QubitRegister(num_qubits) allocates the
 * state.  Allocates 2^n amplitudes of ``dtype`` on the current CUDA device
 * (owned; freed by iqs_destroy) plus small scratch for reductions, and sets
 * the state to |0...0>.  ``stream`` is a cudaStream_t or NULL (legacy default
 * stream).  n in [1, IQS_MAX_QUBITS].  Errors: IQS_EINVAL, IQS_ENOMEM, IQS_ECUDA. */
iqs_status iqs_create(int n, int dtype, void* stream, iqs_reg** out);

/* Section 2 "Scope and basic use" (QubitRegister holds the state), with the
 * storage supplied by the caller; the paper has no call of this form.  Same as
 * iqs_create but borrows ``device_ptr`` (2^n amplitudes of ``dtype``,
 * 16-byte aligned, on the current device), e.g. a torch tensor's storage.
 * The contents are not modified; iqs_destroy never frees the borrowed buffer,
 * and the caller keeps it alive while the register exists. */
iqs_status iqs_wrap(int n, int dtype, void* device_ptr, void* stream, iqs_reg** out);

/* End of a QubitRegister's lifetime (Section 2 "Scope and basic use"): frees
 * what the register owns (synchronising its stream first).  NULL is OK. */
iqs_status iqs_destroy(iqs_reg* reg);

/* Device address of the amplitudes, number of qubits, dtype. */
iqs_status iqs_data(const iqs_reg* reg, void** device_ptr);
iqs_status iqs_info(const iqs_reg* reg, int* n, int* dtype);

/* Stream on which later calls are ordered (cudaStream_t or NULL). */
iqs_status iqs_set_stream(iqs_reg* reg, void* stream);

/* Arithmetic mode of complex128 gates (an iqs_math value); ignored for complex64. */
iqs_status iqs_set_math(iqs_reg* reg, int math);

/* Gate fusion on the register path (the tiles of Section 2's one-qubit gate
 * equation applied several gates at a time).  With ``on`` != 0, iqs_apply_1q
 * on a qubit below 12 (complex64) or 11 (complex128) only queues the gate:
 * the gates queued on a qubit are multiplied in FP64 on the host, and all
 * queued products run as ONE pass over the state (shared-memory tiles of
 * 2^12 / 2^11 amplitudes, register rounds) when anything else touches the
 * register: any other gate or reduction, iqs_data, iqs_download,
 * iqs_synchronize, iqs_set_stream, iqs_set_math, iqs_destroy or iqs_flush
 * (iqs_init_* and iqs_upload discard the queue: the state is replaced).  A
 * caller that reads the device buffer by other means (a wrapped torch
 * tensor) must call iqs_flush first.  Gates on higher qubits run at once,
 * after a flush.  Queued gates are not queued for complex128 with
 * IQS_MATH_NATIVE.  ``on`` = 0 flushes and stops queueing (the default). */
iqs_status iqs_set_fusion(iqs_reg* reg, int on);
iqs_status iqs_flush(iqs_reg* reg);

/* Block the host until the register's stream is idle; reports IQS_ERANGE if
 * an emulated complex128 gate met an out-of-range amplitude since the last
 * check (the flag is cleared by the check). */
iqs_status iqs_synchronize(iqs_reg* reg);

/* ------------------------------------------------------------ state set-up */

/* Section 2 "Scope and basic use", Initialize("base", index): |index>. */
iqs_status iqs_init_basis(iqs_reg* reg, uint64_t index);

/* Section 2 "Scope and basic use", balanced superposition: every amplitude 2^(-n/2). */
iqs_status iqs_init_uniform(iqs_reg* reg);

/* Copy ``bytes`` (must equal 2^n x amplitude size) between a host buffer and
 * the register; synchronous.  Pinned host memory gives full bandwidth. */
iqs_status iqs_upload(iqs_reg* reg, const void* host, size_t bytes);
iqs_status iqs_download(const iqs_reg* reg, void* host, size_t bytes);

/* Stream-ordered partial copies: amplitudes [first, first + count) between a
 * host buffer and the register, asynchronous on the register's stream (host
 * memory must be pinned for the copy to overlap other work, and must stay
 * valid until the stream has passed the copy).  With several streams (one
 * register on a copy stream, registers wrapping slices of the same state on
 * a compute stream, ordered by events) a caller can start the gates that act
 * inside one slice while the next slice is still arriving.  IQS_EINVAL for a
 * NULL buffer or a range outside the state.  Copying in discards queued
 * (iqs_set_fusion) gates; copying out flushes them first. */
iqs_status iqs_copy_to_device(iqs_reg* reg, const void* host, uint64_t first, uint64_t count);
iqs_status iqs_copy_to_host(iqs_reg* reg, void* host, uint64_t first, uint64_t count);

/* Checkpoint and resume (the paper has no such call): write the register's
 * state to ``path`` (the 8 bytes "IQSSTATE", uint32 version 1, n, dtype and a
 * zero word, then the 2^n amplitudes as stored), and read such a file back
 * into a register of the same n and dtype (IQS_EINVAL otherwise, or for a
 * file that is not a state file or is truncated; the register is then
 * unspecified).  Synchronous; staged through a 64 MiB pinned buffer. */
iqs_status iqs_save(iqs_reg* reg, const char* path);
iqs_status iqs_load(iqs_reg* reg, const char* path);

/* ------------------------------------------------------------ gates */

/* Section 2 "Distributed implementation", the one-qubit gate equation:
 * for every index i with i_q = 0, (alpha_i, alpha_{i+2^q}) <- U (alpha_i, alpha_{i+2^q}).
 * q in [0, n).  U may be any 2x2 complex matrix (the paper's "random 2x2
 * matrix"); matrices whose entries are all 0, +-1 or +-i and that have one
 * nonzero per row and column (X, Y, Z, S, ...) are applied exactly. */
iqs_status iqs_apply_1q(iqs_reg* reg, int q, const double U[8]);

/* Section 2 "Scope and basic use" and "Distributed implementation", last
 * paragraph: controlled one-qubit gate, U applied to target t on the basis
 * states whose control bit c is 1 (CNOT = ApplyCPauliX with U = X).
 * c, t in [0, n), c != t. */
iqs_status iqs_apply_c1q(iqs_reg* reg, int c, int t, const double U[8]);

/* Section 2 footnote on the QAOA-specialised methods (one global diagonal
 * operation per step) and Section 4 (H_MaxCut counts the cut edges):
 *   psi_x <- exp(-i gamma C(x)) psi_x,  C(x) = sum_{(u,v)} w_uv (x_u XOR x_v).
 * ``edges``: host int32 array of 2*n_edges vertex indices (u0, v0, u1, v1, ...),
 * each in [0, n), u != v.  ``weights``: host array of n_edges doubles or NULL
 * for weight 1 (the unweighted case uses an FP64-built table of
 * exp(-i gamma k), k = 0..n_edges).  0 <= n_edges <= 4096. */
iqs_status iqs_apply_zz_phase(iqs_reg* reg, int n_edges, const int32_t* edges,
                              const double* weights, double gamma);

/* Section 2 "Scope and basic use": custom gates on several qubits.  A dense
 * 2^k x 2^k matrix U acts on qubits[0..k); bit j of U's row and column index
 * is the value of qubits[j].  ``U`` is row-major, (re, im) doubles: entry
 * (row, col) at U[2 * (row * 2^k + col)].  k: 1..5 for IQS_C64 (computed in
 * FP32), 1..5 for IQS_C128 (double-float emulation or native FP64 as for
 * iqs_apply_1q; with the emulation, k = 3..5 run by default as exact bf16
 * digit products on the tcgen05 tensor cores, an FP64-accurate
 * contraction).  The qubits must be distinct and in [0, n); U must be
 * finite.  IQS_EINVAL otherwise, with the state untouched.  Asynchronous. */
iqs_status iqs_apply_kq(iqs_reg* reg, int k, const int* qubits, const double* U);

/* Project autotuner of iqs_apply_kq: times every kernel variant (0 the fixed
 * rule, 1 shared-memory tiles for targets below bit 5, 2 one group per thread
 * with U in constant memory, 3 rolled rows with U in shared memory, and for
 * emulated complex128 with k = 2..5 also 4, the tensor-core product of exact
 * bf16 digit slices) at 4, 8, 16 and 32 blocks per SM (variant 4: one block
 * per SM), on this register's state with these targets,
 * applying U and its conjugate transpose alternately (an even number of
 * times, so the state comes back up to rounding: U must be unitary), and keeps
 * the fastest for every later iqs_apply_kq of the same dtype, arithmetic, k
 * and target class (a target below bit 5, or none) in this process.  With
 * IQS_AUTOTUNE_CACHE=<file> the choice is appended there and read back by
 * later processes.  A variant that does not apply to a shape falls back to
 * the fixed rule.  Outputs (may be NULL): the time of one gate with the
 * choice, the variant, the blocks per SM. */
iqs_status iqs_kq_autotune(iqs_reg* reg, int k, const int* qubits, const double* U, double* best_ms, int* variant,
                           int* blocks_per_sm);

/* Sets, without timing, the variant (0..4 as for iqs_kq_autotune; a variant
 * that does not apply to a shape falls back to the fixed rule) and blocks per
 * SM (1..64) used by every later iqs_apply_kq of this register's dtype,
 * arithmetic, k and target class in this process.  The paper names no such
 * call (a tuning control of this library).  IQS_EINVAL for a bad k, qubit
 * set, variant or block count. */
iqs_status iqs_kq_set_variant(iqs_reg* reg, int k, const int* qubits, int variant, int blocks_per_sm);

/* ------------------------------------------------------------ reductions (FP64 results, synchronous) */

/* Section 2 "Scope and basic use", GetProbability(q): sum of |alpha_i|^2 over
 * i with bit q set (the raw sum; the state is not renormalised first). */
iqs_status iqs_probability(iqs_reg* reg, int q, double* out);

/* Section 2 "Scope and basic use", GetProbability for every qubit in one
 * read of the state: out[q] for q in [0, n). */
iqs_status iqs_probabilities(iqs_reg* reg, double* out);

/* Section 2 "Scope and basic use": expectation of a product of Pauli matrices,
 * Re <psi| P |psi>.  ``pauli`` is a NUL-terminated string of length n over
 * {I, X, Y, Z}; character k acts on qubit k. */
iqs_status iqs_expectation(iqs_reg* reg, const char* pauli, double* out);

/* Section 2 "Scope and basic use" (expectation of a product of Pauli
 * matrices), the product given by bit masks: bit k of ``xmask`` and ``zmask``
 * marks an X (x only), Z (z only) or Y (both) on qubit k.  Bits at or above n
 * must be zero. */
iqs_status iqs_expectation_masks(iqs_reg* reg, uint64_t xmask, uint64_t zmask, double* out);

/* Section 2 "Scope and basic use": measuring qubits in groups gives the joint
 * statistics of their outcomes.  out[m] (m in [0, 2^k)) = sum of |alpha_i|^2
 * over the indices whose bit qubits[j] equals bit j of m; raw sums, not
 * divided by the norm.  k: 1..min(n, 10), distinct qubits; ``out`` is a host
 * array of 2^k doubles.  Temporary device memory (about 8 x 2^k x 608
 * bytes) is taken from the stream-ordered allocator and returned. */
iqs_status iqs_marginal(iqs_reg* reg, int k, const int* qubits, double* out);

/* Sampling counterpart of measuring all qubits: for each of ``shots`` host
 * uniforms u in [0, 1), out[s] = the first index i whose cumulative weight
 * sum_{j <= i} |alpha_j|^2 exceeds u times the total weight (a zero-weight
 * index is never returned: where rounding leaves u * total at or above the
 * last cumulative value, the last index of nonzero weight).  Cumulative
 * weights: FP64 between chunks of 65536 amplitudes, double-float (about
 * 2^-44 of a chunk's weight) inside a chunk; the rounding order differs
 * from a sequential sum only by rounding.  IQS_EINVAL for a
 * u outside [0, 1), NULL arrays, or a state of zero weight.  Temporary
 * device memory: N / 256 + 2 N / 65536 doubles plus 16 bytes per shot. */
iqs_status iqs_sample(iqs_reg* reg, uint64_t shots, const double* uniforms, uint64_t* out);

/* Squared norm sum_i |alpha_i|^2: the sum of all outcome probabilities of
 * Section 2's GetProbability over the basis states, 1 for a normalised state. */
iqs_status iqs_norm2(iqs_reg* reg, double* out);

/* psi <- psi / ||psi|| (norm accumulated in FP64); IQS_EINVAL for a zero state.
 * The paper names no renormalisation call: its probabilities (Section 2,
 * GetProbability) assume a unit-norm state, which this restores after rounding
 * has moved the norm (complex64 gates, long circuits). */
iqs_status iqs_renormalize(iqs_reg* reg);

/* Section 4: <H_MaxCut> = sum_x C(x) |alpha_x|^2 with C as in iqs_apply_zz_phase. */
iqs_status iqs_energy_maxcut(iqs_reg* reg, int n_edges, const int32_t* edges,
                             const double* weights, double* out);

/* ------------------------------------------------------------ QAOA energy and adjoint gradient */

/* Section 4 ("QAOA with swarm particle optimization"): the objective
 * L(theta) = <0| U^dagger H_MaxCut U |0> of QAOA Max-Cut, evaluated for a pool
 * of parameter sets at once (Section 2, "Pool of multiple states": each pool
 * state runs the same circuit with its own parameters).  Circuit:
 * |+>^n, then for l = 1..p the cost phase exp(-i gamma_l C) and the mixer
 * RX(2 beta_l) = exp(-i beta_l X) on every qubit; C(x) counts cut edges.
 * The gradient is the adjoint derivative dE/dtheta = 2 Im <lambda|G|phi>,
 * computed by uncomputing the state with inverse gates (no stored states). */
typedef struct iqs_qaoa iqs_qaoa;

/* Workspace for up to ``batch_max`` parameter sets of an unweighted graph
 * with ``n_edges`` (1..255) edges (host int32 pairs, u != v, in [0, n)) on n
 * qubits (2..34).  Allocates two state vectors per parameter set (phi and
 * lambda), one byte of cut count per basis state, parameter tables and
 * scratch on the current device.  ``stream`` may be NULL (a private stream is
 * created).  Errors: IQS_EINVAL, IQS_ENOMEM, IQS_ECUDA. */
iqs_status iqs_qaoa_create(int n, int dtype, int batch_max, int n_edges, const int32_t* edges, void* stream,
                           iqs_qaoa** out);
iqs_status iqs_qaoa_destroy(iqs_qaoa* q);

/* renorm_every = R > 0 renormalises phi (to 1) and lambda (to its initial norm)
 * every R uncomputed layers, in FP64; use_graphs != 0 (default) replays each
 * (batch, p, gradient) shape from a captured CUDA graph. */
iqs_status iqs_qaoa_set_options(iqs_qaoa* q, int renorm_every, int use_graphs);

/* Engine of energy-only runs (iqs_qaoa_run without gradient outputs): 0
 * (default) and 1 use the tiled passes; 2 keeps every complex64 state of
 * 8..18 qubits resident in the shared memory of a thread-block cluster for
 * all p layers (up to 16 CTAs of 128 KB; the state is written once, for
 * iqs_qaoa_download_state).  Mode 2 is IQS_EINVAL where it is unavailable.
 * Gradient runs and complex128 always use the tiled passes.  Energies agree
 * within complex64 rounding.  (Measured, the cluster engine ties the tiled
 * passes up to 14 qubits and is slower at 16 and 18, hence the default.) */
iqs_status iqs_qaoa_set_engine(iqs_qaoa* q, int engine);

/* Section 4's L(theta) and its adjoint gradient for a pool of parameter sets
 * (Section 2, "Pool of multiple states").
 * Evaluate ``batch`` parameter sets of depth p (1..64).  Host arrays,
 * row-major [batch][p]: gammas, betas.  Outputs (host): energies[batch] and,
 * when both are non-NULL, grad_gammas[batch][p] and grad_betas[batch][p].
 * Energies and gradients are divided by the computed state's squared norm
 * (FP64), i.e. Rayleigh quotients <phi|C|phi>/<phi|phi>: this removes the
 * norm drift that FP32-rounded gate coefficients leave in complex64 (the norm
 * is 1 in exact arithmetic).  With renorm_every > 0, phi is restored to that
 * norm and lambda to its initial norm.
 * Synchronous.  IQS_ERANGE if a complex128 amplitude left the emulated range. */
iqs_status iqs_qaoa_run(iqs_qaoa* q, int batch, int p, const double* gammas, const double* betas,
                        double* energies, double* grad_gammas, double* grad_betas);

/* Stream-ordered variant of iqs_qaoa_run for callers whose parameters and
 * results live in device memory (a training loop, a batched optimiser): the
 * same evaluation (Section 4's L(theta) and its adjoint gradient for a pool of
 * parameter sets), enqueued on the workspace's stream without any host
 * synchronisation or host copy.  ``d_gammas`` and ``d_betas`` are DEVICE
 * arrays [batch][p]; the outputs ``d_energies`` [batch] and, when both are
 * non-NULL, ``d_grad_gammas`` and ``d_grad_betas`` [batch][p] are DEVICE
 * arrays written on the stream.  The RX coefficients and phase tables are
 * built on the device from the parameters (FP64).  Every pointer must stay
 * valid until the stream has passed the call.  Non-finite parameters are not
 * checked (they give non-finite results); a complex128 range error or a TMA
 * wait that gave up is reported by iqs_qaoa_synchronize.  IQS_EINVAL for bad
 * sizes or NULL outputs, IQS_ECUDA for a failed launch. */
iqs_status iqs_qaoa_run_async(iqs_qaoa* q, int batch, int p, const double* d_gammas, const double* d_betas,
                              double* d_energies, double* d_grad_gammas, double* d_grad_betas);

/* Block until the workspace's stream is idle; IQS_ERANGE if a complex128
 * amplitude left the emulated range, IQS_ETIMEOUT if a TMA wait gave up, in
 * the evaluations since the last check (the flags are cleared). */
iqs_status iqs_qaoa_synchronize(iqs_qaoa* q);

/* Project autotuner: times the pass schedule (chained, or per layer with TMA
 * staging off / forward / forward + adjoint), then the candidate mixer tile
 * shapes (the row width of the high passes,
 * hence gate bits per pass: 4..6 row bits for complex64, 3..5 for complex128)
 * and grid sizes (1x, 2x blocks per state) on this workspace
 * for ``batch`` parameter sets of depth p, and keeps the fastest (every shape
 * gives the same results up to rounding).  With IQS_AUTOTUNE_CACHE=<file> the
 * choice is appended to that file, and later workspaces of the same dtype, n
 * and batch_max start from it.  ``best_ms`` (may be NULL): time of one
 * evaluation of the batch with the chosen shape. */
iqs_status iqs_qaoa_autotune(iqs_qaoa* q, int batch, int p, double* best_ms);

/* Current tile-shape choice: high-pass row bits and grid multiplier. */
iqs_status iqs_qaoa_tuning(const iqs_qaoa* q, int* row_bits, int* grid_mult);

/* Mixer-tile staging by the Tensor Memory Accelerator (cp.async.bulk.tensor
 * loads and stores, double-buffered): mode 0 off, 1 forward passes, 2 forward
 * and adjoint passes.  It applies to full 2^K-amplitude tiles (n >= 12 for
 * complex64, 11 for complex128); ``available`` reports whether the tensor maps
 * of the current plan could be built.  The default is 1; the autotuner also
 * chooses this mode. */
iqs_status iqs_qaoa_set_tma(iqs_qaoa* q, int mode);
iqs_status iqs_qaoa_get_tma(const iqs_qaoa* q, int* mode, int* available);

/* Pass schedule of the tiled engine.  0 (default): chained segments.  The
 * RX factors of a mixer commute and the cost phase is diagonal, so layer l
 * visits its tile passes forwards when l is even and backwards when l is odd;
 * the last pass of one layer, the next layer's phase and that layer's first
 * pass then run in one tile residency.  The turnaround (energy, lambda = C phi)
 * and the first adjoint pass share the forward's last tile, the first pass
 * starts from |+> generated on chip, and the last adjoint pass stores nothing.
 * With m tile passes per mixer a gradient evaluation moves each vector
 * 3 p (m - 1) + 1 times instead of 3 p m + 2.  It needs every pass to be a full
 * tile (n >= 12 for complex64, 11 for complex128); elsewhere, and with
 * schedule 1, one pass sequence per layer runs, with the energy and lambda in
 * a pass of their own (this schedule alone uses TMA staging).  With one pass
 * per mixer the whole evaluation is one tile residency, and renorm_every has
 * no effect.  ``chained_available`` (may be NULL) reports whether the current
 * plan can run chained.  Results agree within rounding. */
iqs_status iqs_qaoa_set_schedule(iqs_qaoa* q, int schedule);
iqs_status iqs_qaoa_get_schedule(const iqs_qaoa* q, int* schedule, int* chained_available);

/* Copy the state phi of parameter set ``index`` to host memory: after an
 * energy-only run, the final state.  After a run with a gradient on the
 * chained schedule the vector holds an intermediate state of the uncompute
 * (the last adjoint pass stores nothing); on schedule 1, the uncomputed state. */
iqs_status iqs_qaoa_download_state(iqs_qaoa* q, int index, void* host, size_t bytes);

/* Several graphs in one workspace (Section 4: the swarm experiment averages
 * over many random 3-regular graphs).  ``edges`` holds n_graphs x n_edges
 * int32 pairs, graph-major; every graph has the same number of edges.  The
 * workspace holds n_graphs x per_graph states (at most 65535); in
 * iqs_qaoa_run, parameter set b is scored on graph b / per_graph.
 * iqs_qaoa_create(n, dtype, B, ...) is the one-graph case. */
iqs_status iqs_qaoa_create_multi(int n, int dtype, int n_graphs, int per_graph, int n_edges, const int32_t* edges,
                                 void* stream, iqs_qaoa** out);

/* Shape of a workspace (any pointer may be NULL).  For a one-graph
 * workspace, per_graph is its batch_max. */
iqs_status iqs_qaoa_info(const iqs_qaoa* q, int* n, int* dtype, int* n_graphs, int* per_graph, int* n_edges);

/* Section 4: E_exact, the exact Max-Cut value of each graph, as the largest
 * cut count over all 2^n bipartitions (read from the workspace's cut
 * tables).  ``out``: host array of n_graphs doubles.  Synchronous. */
iqs_status iqs_qaoa_max_cut(iqs_qaoa* q, double* out);

/* Section 4, "QAOA with swarm particle optimization": particle swarm
 * maximisation of L(theta) = <H_MaxCut>, theta = (gamma_1..gamma_p,
 * beta_1..beta_p), one swarm of per_graph particles per graph of the
 * workspace, all swarms scored together in one iqs_qaoa_run per step
 * (energies only).  Each step, for particle k of graph g:
 *   v <- omega v + phi_p r_p (theta_best_k - theta) + phi_g r_g (theta_best_g - theta),
 *   theta <- theta + v,
 * then every new position is scored; a particle's best (and then the swarm's
 * best) moves only to a strictly larger score, and the swarm's best used by a
 * step is the one after the previous step.  Reading: the paper's printed
 * velocity update has theta - theta_best in both attraction terms, which
 * would repel the particles; the standard swarm update (Kennedy and
 * Eberhart 1995), which attracts them, is taken.  r_p and r_g are one number
 * per particle per step, as the paper's equation writes them.
 *
 * Host arrays (G = n_graphs, R = per_graph):
 *   pos0, vel0  [G][R][2p]           initial positions and velocities
 *   rp, rg      [steps][G][R]        the uniform draws
 *   trace       [G][(steps+1) R]     best score so far after each evaluation
 *                                    (step-major, particles in order)
 *   best_pos    [G][2p], best_val [G]
 * All random numbers are inputs.  Scores are the engine's energies (complex64
 * or complex128, as created). */
iqs_status iqs_qaoa_pso(iqs_qaoa* q, int p, int steps, const double* pos0, const double* vel0, const double* rp,
                        const double* rg, double omega, double phi_p, double phi_g, double* trace, double* best_pos,
                        double* best_val);

/* ------------------------------------------------------------ pool of noisy trajectories */

/* Section 2 "Pool of multiple states" and the pool-of-states appendix: a pool
 * of states runs the same circuit, each with its own stochastic noise
 * rotations, and a probability is averaged incoherently over the pool (sum
 * over the pool's states divided by their number).
 * Circuit family ("brick"): layer l applies U[l][q] to every qubit q, then
 * CNOT(i, i+1) for i = o, o + 2, ... (o = l mod 2, i + 1 < n).  With noise,
 * each gate is followed, on every qubit it touched (the target of a one-qubit
 * gate; control then target of a CNOT), by RX(tx) then RZ(tz),
 * R(t) = exp(-i t sigma / 2), with angles that differ per trajectory. */
typedef struct iqs_pool iqs_pool;

/* Workspace for up to ``batch_max`` trajectories of n qubits (2..24) and
 * circuits of up to ``depth_max`` layers, on the current device. */
iqs_status iqs_pool_create(int n, int dtype, int batch_max, int depth_max, void* stream, iqs_pool** out);
iqs_status iqs_pool_destroy(iqs_pool* p);

/* Number of noise rotations (angle pairs) per trajectory of a depth-layer
 * brick circuit on n qubits: sum over layers of n + 2 x (CNOTs in the layer). */
int iqs_pool_noise_count(int n, int depth);

/* Noise gates from relaxation and dephasing times (Section 2 and the pool
 * appendix: SetNoiseTimescales(T1, T2), ApplyNoiseGate(qubit, duration)).
 * After this call, every noise rotation of iqs_pool_run_brick is a noise
 * gate of duration ``gate_time``: RX(s_x z_x), then RY(s_y z_y), then
 * RZ(s_z z_z), and ``angles`` holds the standard normal draws
 * [batch][iqs_pool_noise_count(n, depth)][3] = (z_x, z_y, z_z).  The
 * deviations are s_x^2 = s_y^2 = t / T1 and s_z^2 = 2 t / T2 - t / T1, so the
 * gate averaged over its draws is the Pauli-twirled relaxation and dephasing
 * channel: Bloch components transverse to Z decay by exp(-t / T2), the Z
 * component by exp(-t / T1).  (The paper cites other work for the angle law;
 * this is the reading.)  Needs 0 < T2 <= 2 T1 and gate_time >= 0; T1 <= 0
 * returns to the (tx, tz) angle pairs. */
iqs_status iqs_pool_set_noise_t1t2(iqs_pool* p, double T1, double T2, double gate_time);

/* Execution engine of iqs_pool_run_brick: 0 (default) picks the
 * cluster-resident engine when a state fits, 1 forces the tiled passes
 * (two passes over every state per layer through HBM), 2 forces the
 * cluster-resident engine: each trajectory lives in the distributed shared
 * memory of a thread-block cluster (up to 16 CTAs of 128 KB) for the whole
 * circuit, and its state is written to HBM once at the end.  It takes
 * complex64 states of 8..18 qubits and complex128 of 8..17 (clusters of up
 * to 16 CTAs); mode 2 on a state that does not fit is IQS_EINVAL.  Mode 0
 * uses it for complex64 states that fit clusters of up to 4 CTAs (16
 * qubits).  Results agree within the
 * rounding of the dtype (the gates are grouped differently). */
iqs_status iqs_pool_set_engine(iqs_pool* p, int engine);

/* Project autotuner of the pool engine: times the tiled passes and the
 * cluster-resident engine at every cluster size that can hold the state
 * (2^logc CTAs, from the smallest that fits up to 16) on ``batch``
 * trajectories of a ``depth``-layer brick circuit (noisy or not), keeps the
 * fastest for this pool (iqs_pool_set_engine is overridden) and, with
 * IQS_AUTOTUNE_CACHE=<file>, appends it there; pools created later with the
 * same dtype, n and batch_max start from it.  ``best_ms`` (may be NULL): time
 * of one run with the choice.  Results agree within the dtype's rounding
 * whatever the choice. */
iqs_status iqs_pool_autotune(iqs_pool* p, int batch, int depth, int noisy, double* best_ms);

/* Current engine (1 tiled passes, 2 cluster-resident, 0 automatic) and
 * cluster size exponent (-1: the smallest that holds the state). */
iqs_status iqs_pool_tuning(const iqs_pool* p, int* engine, int* logc);

/* Section 2 "Pool of multiple states": run ``batch`` trajectories of one
 * brick circuit from |0...0>, each with its own noise rotations, and average
 * P(q = 1) over the pool.  ``unitaries``: host doubles
 * [depth][n][8] (each U row-major as (re, im) pairs).  ``angles``: host
 * doubles [batch][iqs_pool_noise_count(n, depth)][2] = (tx, tz) in the order
 * the rotations occur (layer by layer: the one-qubit gates q = 0..n-1, then
 * each CNOT's control and target), or NULL for the noiseless circuit.
 * Outputs (host): probs[batch][n] = P(q = 1) of each trajectory (divided by
 * the computed state's squared norm, FP64) or NULL; mean[n] = pool average.
 * Synchronous.  On the tiled passes the first run of each (batch, depth,
 * noisy) shape is captured as a CUDA graph and later runs of that shape replay
 * it (the inputs sit in fixed device buffers); iqs_pool_set_noise_t1t2 drops
 * the captured graphs.  A pool on the legacy default stream launches directly. */
iqs_status iqs_pool_run_brick(iqs_pool* p, int batch, int depth, const double* unitaries, const double* angles,
                              double* probs, double* mean);

/* Stream-ordered variant of iqs_pool_run_brick (Section 2 "Pool of multiple
 * states"; the same circuit family, noise model and results) for inputs and
 * outputs in device memory: ``d_unitaries`` [depth][n][8] and ``d_angles``
 * (pairs or T1/T2 triples per trajectory, or NULL) are DEVICE arrays, copied
 * on the pool's stream into its buffers; ``d_probs`` [batch][n] (or NULL) and
 * ``d_mean`` [n] are DEVICE arrays written on the stream.  No host
 * synchronisation; every pointer must stay valid until the stream has passed
 * the call.  A complex128 range error is reported by iqs_pool_synchronize. */
iqs_status iqs_pool_run_brick_async(iqs_pool* p, int batch, int depth, const double* d_unitaries,
                                    const double* d_angles, double* d_probs, double* d_mean);

/* Block until the pool's stream is idle; IQS_ERANGE if a complex128 amplitude
 * left the emulated range since the last check (the flag is cleared). */
iqs_status iqs_pool_synchronize(iqs_pool* p);

/* Copy trajectory ``index``'s final state to host memory. */
iqs_status iqs_pool_download_state(iqs_pool* p, int index, void* host, size_t bytes);

/* A pool of brick circuits of uneven qubit counts, depths and trajectory
 * counts, run in ONE persistent kernel launch (Section 2 "Pool of multiple
 * states"; same circuit family and noise model as iqs_pool_run_brick). */
typedef struct iqs_circuit_desc {
  int n;                    /* qubits, 2..24 */
  int depth;                /* brick layers, >= 1 */
  int trajectories;         /* pool states of this circuit (1 when angles is NULL) */
  const double* unitaries;  /* host [depth][n][8] */
  const double* angles;     /* host [trajectories][iqs_pool_noise_count(n, depth)][2], or NULL */
} iqs_circuit_desc;

typedef struct iqs_pool_many iqs_pool_many;

/* Workspace; device memory is allocated (and kept, growing) by the runs. */
iqs_status iqs_pool_many_create(int dtype, void* stream, iqs_pool_many** out);
iqs_status iqs_pool_many_destroy(iqs_pool_many* w);

/* Every wait inside the persistent kernel gives up after ``seconds`` (default
 * 2): the kernel then stops all its blocks and the run returns IQS_ETIMEOUT
 * with the GPU context intact.  ``debug_never`` != 0 is a test mode in which
 * the first job's first wait can never be satisfied, so the timeout path runs. */
iqs_status iqs_pool_many_set_wait_limit(iqs_pool_many* w, double seconds, int debug_never);

/* Engine of iqs_pool_many_run: 0 (default) runs every trajectory of every
 * circuit in one launch of the cluster-resident engine (see
 * iqs_pool_set_engine) when the dtype is complex64 and every state fits one
 * cluster size of up to 4 CTAs (qubit counts from 2 logc + 1 to the
 * largest), else the
 * persistent tiled kernel; 1 forces the persistent kernel (the only one with
 * bounded waits and IQS_ETIMEOUT); 2 forces the cluster-resident engine
 * (IQS_EINVAL at run time when a state does not fit). */
iqs_status iqs_pool_many_set_engine(iqs_pool_many* w, int engine);

/* Run all circuits (at most 8 distinct qubit counts per call) from |0...0>.
 * Outputs (host): probs = per-trajectory P(q = 1) (divided by the state's FP64
 * squared norm), concatenated circuit by circuit as [trajectories][n], or NULL;
 * means = per-circuit pool averages, concatenated as [n].  Synchronous. */
iqs_status iqs_pool_many_run(iqs_pool_many* w, int n_circuits, const iqs_circuit_desc* circuits, double* probs,
                             double* means);

/* Pools of circuits given as gate lists (Section 2 "Pool of multiple states":
 * every pool state runs its own circuit; noise gates are one-qubit rotations
 * with stochastic angles).  An op applies the 2x2 matrix U (row-major,
 * (re, im) pairs, as iqs_apply_1q) to ``target``, or, with control >= 0, to
 * the target of the basis states whose ``control`` qubit is 1 (as
 * iqs_apply_c1q; CNOT = U = X).  Ops act in order. */
typedef struct iqs_op {
  int control;  /* -1: one-qubit gate; else the control qubit, != target */
  int target;
  double U[8];
} iqs_op;

typedef struct iqs_ops_circuit {
  int n;                 /* qubits, 2..24 */
  int n_ops;
  const iqs_op* ops;     /* host array of n_ops ops */
  int trajectories;      /* pool states of this circuit (1 when angles is NULL) */
  const double* angles;  /* host [trajectories][iqs_ops_noise_count(n_ops, ops)][2], or NULL (noiseless) */
} iqs_ops_circuit;

/* Noise rotations per trajectory of a gate list: after every op, each qubit
 * it touched (the target; the control, then the target) gets RX(tx) then
 * RZ(tz), R(t) = exp(-i t sigma / 2); the count is the number of one-qubit ops
 * plus twice the number of controlled ops (-1 for a bad argument). */
int iqs_ops_noise_count(int n_ops, const iqs_op* ops);

/* Run every trajectory of every gate-list circuit from |0...0> in one launch
 * (one CTA per trajectory; each state in shared memory when it fits, 2^14
 * complex64 or 2^13 complex128 amplitudes, else in an L2-resident slot of the
 * workspace).  The ops are compiled once per circuit: noise rotations fuse
 * into the one-qubit matrix before them, consecutive one-qubit matrices on a
 * qubit fuse, and commuting steps are packed into register rounds of 4
 * (complex64) or 3 (complex128) target bits.  Outputs (host), as for
 * iqs_pool_many_run: probs = per-trajectory P(q = 1) divided by the state's
 * squared norm, concatenated circuit by circuit as [trajectories][n], or NULL;
 * means = per-circuit pool averages, concatenated as [n].  Synchronous.
 * IQS_EINVAL for a qubit out of range, control == target, a non-finite
 * matrix entry or bad sizes. */
iqs_status iqs_pool_many_run_ops(iqs_pool_many* w, int n_circuits, const iqs_ops_circuit* circuits, double* probs,
                                 double* means);

/* ------------------------------------------------------------ allocation-free variant */

/* The paper has no counterpart to this call: it is an interface for callers
 * that cannot call cudaMalloc (an allocator that owns all device memory, a
 * loop that must not allocate after start-up).  It computes what
 * iqs_probabilities computes -- P(q = 1) for every qubit in one read -- from a
 * caller-owned state and writes the n results to a caller-owned DEVICE array,
 * without a register and without allocating anything.
 *   state   device pointer to 2^n amplitudes of ``dtype`` (16-byte aligned).
 *   n       number of qubits, 1..IQS_MAX_QUBITS; anything else is rejected
 *           with IQS_EINVAL (the fixed scratch is sized for at most 34 qubits).
 *   stream  cudaStream_t or NULL; the call is asynchronous on it.
 *   out     device pointer to n doubles (8-byte aligned), written on ``stream``;
 *           all NaN if a complex128 amplitude was outside the emulated range.
 * Scratch is one static device array of about 320 KiB that every GPU loading
 * the library keeps until exit.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress), so make that first call
 * before any stream capture on that device.  The address is cached with the
 * id of the CUDA context it belongs to; after the context is destroyed and
 * created again (cudaDeviceReset), the next call looks it up again, and that
 * call too should precede any capture.  All calls share the array: calls
 * that overlap on the GPU race and must be ordered by the caller.
 * Never calls cudaMalloc, cudaFree or any allocating routine. */
iqs_status iqs_probabilities_noalloc(const void* state, int n, int dtype, void* stream, double* out);

/* ------------------------------------------------------------ diagnostics */

/* Message for the last failed call on this thread ("" if none). */
const char* iqs_last_error(void);

/* Library version string. */
const char* iqs_version(void);

/* Number of CUDA kernels this library has launched in this process (all
 * registers, all threads); for launch accounting in benchmarks. */
uint64_t iqs_kernel_launches(void);

/* Host-side fault injection, for testing error paths without any GPU fault.
 * kind 1: the (after + 1)-th next device allocation of iqs_create, iqs_wrap,
 * iqs_qaoa_create or iqs_pool_create fails with IQS_ENOMEM; kind 2: the
 * (after + 1)-th next kernel-launching call fails with IQS_ECUDA before
 * anything is queued (the state is untouched); kind 0 disarms.  One fault is
 * armed at a time and fires once.  The environment variable IQS_FAULT =
 * "alloc[:after]" or "launch[:after]" arms the same when the library loads. */
iqs_status iqs_inject_fault(int kind, int after);

#ifdef __cplusplus
}
#endif

#endif /* IQS_H */
