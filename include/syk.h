/*
 * libsyk — matrix-free sparse-SYK OTOC path on one B300 (sm_103a).
 *
 * Paper: Garcia-Garcia, Liu, Verbaarschot, "Sparsity independent Lyapunov
 * exponent in the SYK model" (arXiv 2311.00639).  Citations below name the
 * paper's equations, sections and algorithms.
 *
 * ---------------------------------------------------------------------------
 * Conventions (every call)
 *   * N Majoranas, N even, 4 <= N <= 64.  L = N/2 - 1 qubits per parity block,
 *     D = 2^L amplitudes per block.  chi_n = gamma_n / sqrt(2),
 *     {chi_m, chi_n} = delta_mn (main text, below Eq. (1)).
 *   * Qubit s is bit s of a basis index; sigma_y = [[0,-i],[i,0]] (the form
 *     Algorithm 1 implements with coeff = lambda i^{#sigma_y}).
 *   * Representation SYK_REP_PAPER: supplement Eq. (S1), compact form; block
 *     U = top qubit 0, D = top qubit 1; block index m = the other L bits.
 *     gamma_{N-1} has UD = -i, DU = +i; gamma_{N-2} blocks = sigma_z on qubit L-1.
 *   * Representation SYK_REP_JW: gamma_{2s} = Z_0..Z_{s-1} X_s,
 *     gamma_{2s+1} = Z_0..Z_{s-1} Y_s on N/2 qubits; block U = even popcount
 *     of the full index, D = odd; block index m drops the top qubit.  Every
 *     four-Majorana term flips at most four bits of m (best locality).
 *   * A state of one block is D complex numbers (SYK_C64: interleaved float
 *     re,im; SYK_C128: interleaved double re,im), contiguous.  `nstates`
 *     states are stored one after another ([nstates][D]).
 *   * Vector pointers are DEVICE pointers owned by the caller (e.g. torch
 *     tensors); the library never frees caller memory.  Pointers must be
 *     16-byte aligned.  Every call with a cudaStream_t is asynchronous on that
 *     stream unless stated otherwise.
 *   * A complex64 handle keeps a device tile counter that its H psi passes
 *     draw work from and, for blocks of at most ~2^19 amplitudes with many
 *     terms, a workspace for the partial sums of passes split across CTAs;
 *     calls that apply one handle (syk_apply_H, syk_krylov_evolve[_noalloc],
 *     syk_otoc) must therefore not overlap on the GPU: issue them on one
 *     stream, or order the streams with events.  Different handles are
 *     independent.
 *   * Return value: SYK_OK (0) or a negative status.  syk_last_error() gives
 *     the message of the last failing call on the calling thread.  No C++
 *     exception crosses this interface.
 * ---------------------------------------------------------------------------
 */
#ifndef SYK_H
#define SYK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* syk_stream_t; /* == cudaStream_t */

enum {
  SYK_OK = 0,
  SYK_EINVAL = -1,   /* invalid argument */
  SYK_ENOMEM = -2,   /* device or host allocation failed */
  SYK_ENOCONV = -3,  /* Krylov substep control did not converge */
  SYK_ETIMEOUT = -4, /* a bounded device wait expired */
  SYK_ECUDA = -5,    /* CUDA runtime error */
  SYK_EAGAIN = -6    /* no free slot or memory right now (batched engine); retry later */
};
enum { SYK_C64 = 0, SYK_C128 = 1 };
enum { SYK_REP_JW = 0, SYK_REP_PAPER = 1, SYK_REP_PAULI = 2 /* Pauli-string handle (syk_build_pauli_terms) */ };
enum { SYK_BLOCK_U = 0, SYK_BLOCK_D = 1 };
enum { SYK_OTOC_TYPICAL = 0, SYK_OTOC_EXACT_TRACE = 1 };

typedef struct syk_terms syk_terms_t;

/* Summary of a compiled Hamiltonian (host struct). */
typedef struct {
  int N, L, dtype, rep;
  int64_t D;           /* amplitudes per block */
  int64_t n_input;     /* quadruples given */
  int64_t n_terms;     /* Pauli strings after merging duplicates */
  int64_t n_real;      /* strings with a real coefficient (the rest are i * real) */
  int64_t n_xgroups;   /* distinct flip masks */
  double sum_abs_coef; /* sum_t |c_t|, a bound on ||H_block|| */
  int64_t n_passes;    /* matvec passes (term groups with an L2-resident working set) */
  int64_t device_error; /* 1 if a kernel on this handle hit its bounded-wait limit (then results
                           are invalid); reading it synchronises with the device */
  int64_t n_tile_reads; /* input tiles staged per output tile over all passes of one H psi:
                           complex64 terms of a pass that read the same tile share one copy;
                           complex128 stages one tile per term */
  int64_t n_merged;     /* complex64: terms whose body runs with the next term's (same flip mask and
                           class: one body per group of such terms); 0 for complex128 */
} syk_terms_info;

/*
 * syk_build_terms — compile H = sum_t J_t chi_i chi_j chi_k chi_l (Eq. (1)).
 *   quads : HOST int32 [T][4], each row strictly increasing, entries in [0, N).
 *   J     : HOST double [T], chi-normalised couplings (any real values).
 *   dtype : SYK_C64 or SYK_C128 — the state type every later call uses.
 *   rep   : SYK_REP_JW or SYK_REP_PAPER.
 * Each term becomes one Pauli string on the L-qubit block, Phi[m] +=
 * c (-1)^{popc(z & m)} psi[m ^ x], by the operator product rule of the
 * supplement Sec. I.A (XOR of flip masks, phase from the sign pattern);
 * duplicates are merged (supplement Sec. I.A, operator addition).  Terms are
 * grouped by flip mask.  The table is uploaded to the current device; the
 * handle owns it.  T = 0 is allowed (H = 0).  Errors: SYK_EINVAL (bad N,
 * unsorted or out-of-range quad, non-finite J), SYK_ENOMEM, SYK_ECUDA.
 */
int syk_build_terms(int N, int64_t T, const int32_t* quads, const double* J, int dtype, int rep,
                    syk_terms_t** out);
int syk_terms_destroy(syk_terms_t* h);
int syk_terms_get_info(const syk_terms_t* h, syk_terms_info* info);
/*
 * syk_terms_replan — regroup the terms into matvec passes.  Each pass fixes a
 * set of high index bits that its terms do not flip and visits the block one
 * fixed value of those bits at a time ("super-tile"), so that its inputs are
 * re-read from L2; l2_budget_bytes bounds the super-tile size.
 * straggler_ratio > 0 lets the planner dissolve light passes, moving their
 * terms into heavier passes that fetch them from HBM instead; 0 disables it.
 * l2_budget_bytes = 0 restores the default plan of syk_build_terms (the best
 * of a sweep on B300 at N = 64: complex64 32 MiB and ratio 3, complex128
 * 2 MiB and ratio 1.5; straggler_ratio is then ignored).  Synchronises the
 * device and re-uploads the table; results are unchanged up to floating-point
 * summation order.  Not to be called while the handle is in use on a stream.
 * Errors: SYK_EINVAL (l2_budget_bytes in 1..4095, negative or non-finite
 * straggler_ratio).
 */
int syk_terms_replan(syk_terms_t* h, size_t l2_budget_bytes, double straggler_ratio);
/*
 * Copy the compiled table to HOST arrays of length info.n_terms (any may be
 * NULL): flip mask x, sign mask z, coefficient per block (coef_U, coef_D)
 * and imag flag (1 if the coefficient is i * coef).  Matrix element:
 * (H_P psi)[m] = sum_t coef_P[t] * (imag ? i : 1) * (-1)^{popc(z[t] & m)} * psi[m ^ x[t]].
 */
int syk_terms_export(const syk_terms_t* h, uint32_t* x, uint32_t* z, double* coef_U, double* coef_D,
                     uint8_t* imag);

/*
 * Host-only compilation (no CUDA call; usable without a GPU).  Same rules as
 * syk_build_terms.  Writes up to `capacity` strings into the HOST arrays and
 * the true count into *n_terms (arrays may be NULL to query the count).
 */
int syk_compile_terms_host(int N, int64_t T, const int32_t* quads, const double* J, int rep, int64_t capacity,
                           int64_t* n_terms, uint32_t* x, uint32_t* z, double* coef_U, double* coef_D,
                           uint8_t* imag);
/* One matvec pass of a host plan (syk_plan_host). */
typedef struct {
  int32_t t0, ti, t1;   /* terms [t0, t1) of the plan order: [t0, ti) real, [ti, t1) imaginary */
  uint32_t emask;       /* amplitude-index bits that the pass's covered terms do not flip; the
                           pass visits one value of them (a super-tile) at a time */
  int32_t cls[9];       /* terms of class c = 4 imag + 2 (x & 1) + (z & 1) are [cls[c], cls[c+1]) */
  int32_t split_chunks; /* complex64: CTAs that share each output tile (1 = not split) */
  int32_t split_terms;  /* terms per chunk of a split pass (0 if not split) */
  uint32_t dep[3][256]; /* visit order: the pass's b-th tile starts at amplitude
                           dep[0][b & 255] | dep[1][(b >> 8) & 255] | dep[2][(b >> 16) & 255] */
} syk_pass_info;

/* Outputs of syk_plan_host.  The caller sets the capacities and array
 * pointers (HOST memory; any pointer may be NULL); the call sets the counts.
 * Arrays are written only when both capacities cover the counts, so a first
 * call with zero capacities queries the sizes. */
typedef struct {
  int64_t term_capacity, pass_capacity;
  syk_pass_info* passes; /* [pass_capacity] */
  uint32_t* x;           /* [term_capacity], plan order (pass, class, x, z) */
  uint32_t* z;
  double* coef_U;
  double* coef_D;
  uint8_t* imag;
  uint8_t* straggler; /* 1: the term reads outside its pass's super-tile (from HBM) */
  uint32_t* records;  /* [2][n_terms + 1][4]: the complex64 records of block U, then D, as the
                         kernel reads them: x, z, coefficient (float bits), flags */
  int64_t n_terms, n_passes;
  int64_t n_runs;   /* records that start a run (a new staged input tile) */
  int64_t n_merges; /* records flagged "merge with the next" (flags bit 4) */
} syk_plan_host_out;

/*
 * Host-only (no CUDA call): the pass plan and complex64 record layout that
 * syk_build_terms followed by syk_terms_replan(l2_budget_bytes,
 * straggler_ratio) sets up for these terms, on a device with n_sm SMs.
 * Same argument rules as syk_build_terms and syk_terms_replan.  Records
 * within a pass are ordered by (x >> 11, class, x, z); flags bit 0
 * straggler, 1 run start, 2 run end, 3 imaginary coefficient, 4 merge (the
 * next record of the pass has the same x and class: the kernel sums the two
 * terms' coefficients and applies their shared body once), bits 8-13 the
 * consumer body 32 imag + 16 (x & 1) + 8 (z & 1) + ((x >> 6) & 7); bit 31 of
 * flags, x and z hold bits 6, 7 and 8 of z (x and z fit in 31 bits).
 * Errors: SYK_EINVAL.
 */
int syk_plan_host(int N, int64_t T, const int32_t* quads, const double* J, int dtype, int rep,
                  size_t l2_budget_bytes, double straggler_ratio, int n_sm, syk_plan_host_out* out);
/*
 * syk_plan_strings_host — as syk_plan_host for an already compiled list of n
 * block strings on L index bits (1 <= L <= 31; e.g. the output of
 * syk_compile_pauli_host, with coef_U = coef_D = coef, or of
 * syk_compile_terms_complex_host): x, z (below 2^L), coef_U, coef_D, imag
 * are HOST arrays of n.  The plan, split and records are those
 * syk_build_pauli_terms / syk_build_terms_complex upload for these strings.
 * Errors: SYK_EINVAL.
 */
int syk_plan_strings_host(int L, int64_t n, const uint32_t* x, const uint32_t* z, const double* coef_U,
                          const double* coef_D, const uint8_t* imag, int dtype, size_t l2_budget_bytes,
                          double straggler_ratio, int n_sm, syk_plan_host_out* out);
/*
 * Host-only: chi_n from block P as (chi psi)[m] = c_P (-1)^{popc(z & m)} psi[m ^ x]
 * in the other block; c_P = re[P] + i im[P] (arrays of 2).
 */
int syk_compile_chi_host(int N, int rep, int n, uint32_t* x, uint32_t* z, double* re, double* im);

/*
 * syk_apply_H — out = H_PP psi for block P (Algorithm 1, supplement
 * Sec. I.A; K1 of the hot path).  psi, out: [nstates][D] device, dtype of h;
 * out must not overlap psi.  Errors: SYK_EINVAL (null pointer, bad block,
 * overlap, nstates < 1), SYK_ECUDA.
 */
int syk_apply_H(const syk_terms_t* h, int block, const void* psi, void* out, int64_t nstates,
                syk_stream_t stream);

/*
 * syk_apply_chi — out = chi_i psi, mapping block from_block to the other
 * block (supplement, parity-block OTOC formula; for the paper representation
 * chi_{N-1}: U->D times +i/sqrt2, D->U times -i/sqrt2, and chi_{N-2}: sigma_z on
 * qubit L-1 over sqrt2).  For i with an empty flip mask (chi_{N-1}, chi_{N-2}
 * in both representations) out may alias psi; otherwise it must not.
 */
int syk_apply_chi(const syk_terms_t* h, int i, int from_block, const void* psi, void* out,
                  int64_t nstates, syk_stream_t stream);

/*
 * syk_random_state — typical-state amplitudes (supplement: Haar-random
 * state; K4).  Writes UNNORMALISED i.i.d. standard complex Gaussians
 * (E|a|^2 = 2) into psi_U and psi_D (D each).  Amplitude g = block*D + m uses
 * Philox4x32-10 (Salmon et al., SC'11) with counter (g lo, g hi, state_id lo,
 * state_id hi) and key (seed lo, seed hi); words w0..w3 give
 * u1 = ((w1:w0 >> 11) + 1) 2^-53, u2 = (w3:w2 >> 11) 2^-53 and
 * a = sqrt(-2 ln u1) (cos 2 pi u2 + i sin 2 pi u2).  Either pointer may be NULL.
 */
int syk_random_state(const syk_terms_t* h, uint64_t seed, uint64_t state_id, void* psi_U, void* psi_D,
                     syk_stream_t stream);

/* Krylov (Lanczos) propagation parameters.  Zero fields take the defaults. */
typedef struct {
  int m;            /* Krylov dimension per substep (default 20 C64, 30 C128; max 64) */
  double tol;       /* relative error target per evolve (default 1e-12 C128, 1e-6 C64) */
  int max_substeps; /* default 1000 */
  int reorth;       /* 1: full re-orthogonalisation (classical Gram-Schmidt twice) */
  int two_pass;     /* 1: do not store the basis; regenerate it in a second pass */
} syk_krylov_params;

typedef struct {
  int64_t matvecs;
  int64_t substeps;
  double err_est; /* sum of accepted local error estimates (relative) */
} syk_krylov_stats;

/* Bytes of device workspace syk_krylov_evolve needs for these parameters. */
size_t syk_krylov_workspace_bytes(const syk_terms_t* h, const syk_krylov_params* p);

/*
 * syk_krylov_evolve — y = e^{-(tau + i t) H_PP} x for each of nstates states
 * (supplement Sec. I.A: restarted Krylov method for the state time
 * evolution; here Lanczos with an a-posteriori error estimate and substep
 * control in the manner of Expokit, Sidje 1998).  Lanczos scalars (alpha,
 * beta, norms, the tridiagonal eigensystem and exponential) are float64 on
 * the device for both dtypes.  y may alias x.  workspace: device, at least
 * syk_krylov_workspace_bytes().  stats: HOST, may be NULL.  The call returns
 * after the result is complete on `stream` (it synchronises once per
 * substep to read the accepted step).  Errors: SYK_EINVAL, SYK_ENOCONV,
 * SYK_ECUDA.
 */
int syk_krylov_evolve(const syk_terms_t* h, int block, double tau, double t, const void* x, void* y,
                      int64_t nstates, const syk_krylov_params* p, void* workspace, size_t ws_bytes,
                      syk_krylov_stats* stats, syk_stream_t stream);

/*
 * syk_krylov_evolve_noalloc — the same propagation as syk_krylov_evolve
 * (same kernels, same results), for callers that cannot allocate device
 * memory while they run: e.g. a program that embeds this library under
 * another framework's memory pool which already owns the device memory, or a
 * service whose device footprint must stay fixed after start-up.  It takes
 * no workspace argument and allocates nothing; its workspace is a static
 * device array of 16 MiB inside the library, held on every GPU where it has
 * been called (see the first-call rule below) until the process exits.  The paper has no counterpart to this
 * call.
 *   * A call whose workspace (syk_krylov_workspace_bytes with the same
 *     params) exceeds 16 MiB returns SYK_EINVAL without queuing work.
 *   * All calls on a device share the array and leave their contents in it;
 *     calls that overlap on the GPU (other streams, other host threads) race
 *     and corrupt each other's results: serialise them.
 *   * The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, once per device).  CUDA loads the library's
 *     device code lazily, so that first call is also when the 16 MiB are
 *     reserved on the device: it does take device memory.  Callers that must
 *     not allocate later make one warm-up call at start-up, before any
 *     stream capture: tau = t = 0 reserves the array (it only copies x to
 *     y); a real evolve of the kind they will run also loads its kernels.
 *     Later calls allocate nothing.
 *   * The address is cached for the device context current at the first
 *     call; like every handle, it does not survive cudaDeviceReset or a
 *     re-created primary context.
 * Arguments, aliasing, synchronisation and errors are as for
 * syk_krylov_evolve.
 */
int syk_krylov_evolve_noalloc(const syk_terms_t* h, int block, double tau, double t, const void* x, void* y,
                              int64_t nstates, const syk_krylov_params* p, syk_krylov_stats* stats,
                              syk_stream_t stream);

/*
 * syk_otoc — regularised OTOC, Eq. (2), via the parity-block single-state
 * formula of the supplement:
 *   F_P(t) = <psi_P| e^{(it-b/8)H_PP} chi_a e^{-(it+b/4)H_QQ} chi_b
 *            e^{(it-b/4)H_PP} chi_a e^{-(it+b/4)H_QQ} chi_b e^{-bH_PP/8} |psi_P>,
 *   F = F_U + F_D,  OTOC(t) = Re mean_s F_s(t) / Re mean_s F_s(0).
 *   a, b      : Majorana indices (the paper: a = N-1, b = N-2).
 *   t_grid    : HOST double [n_t], non-decreasing, t_grid[0] = 0.
 *   mode      : SYK_OTOC_TYPICAL (states from psi_opt, else from
 *               syk_random_state(seed, s) normalised over both blocks) or
 *               SYK_OTOC_EXACT_TRACE (all 2D basis states; F = Tr[...]/2D).
 *   psi_opt   : optional DEVICE [n_states][2][D] (U block then D block),
 *               used as given (normalise them yourself).
 *   F_raw     : HOST double [n_states][n_t][2] (re, im) per state (exact trace:
 *               n_states is ignored and one row is written), may be NULL.
 *   otoc      : HOST double [n_t], may be NULL.
 * Allocates its own device workspace for the call and frees it before
 * returning; blocks until the host outputs are written.
 */
int syk_otoc(const syk_terms_t* h, int a, int b, double beta, const double* t_grid, int n_t, int mode,
             int n_states, uint64_t seed, const void* psi_opt, const syk_krylov_params* p, double* F_raw,
             double* otoc, syk_krylov_stats* stats, syk_stream_t stream);

/*
 * ---------------------------------------------------------------------------
 * Pauli-string (spin-chain) Hamiltonians.  The paper's conclusions name OTOCs
 * of sparse spin chains, such as those of many-body-localisation studies, as
 * the next use of its GPU machinery; the supplement (Sec. I.A) stores every
 * operator as a list of Pauli strings with coefficients.  These calls take
 * such a list directly, H = sum_t h_t P_t on n_qubits qubits, and run it
 * through the same H psi, Krylov and OTOC kernels as the SYK handles.
 *   * A string is two masks: on qubit q (bit q of a basis index), x_q alone
 *     = sigma_x, z_q alone = sigma_z, both = sigma_y = [[0,-i],[i,0]]; no bit
 *     = identity.  h_t is real, so H is Hermitian.  With k = popc(x & z),
 *     P = i^k X^x Z^z and (P psi)[m] = (-i)^k (-1)^{popc(z & m)} psi[m ^ x].
 *   * The handle's state space is all 2^n_qubits amplitudes: D = 2^n_qubits,
 *     L = n_qubits.  It holds no Majoranas (info.N = 0, info.rep =
 *     SYK_REP_PAULI), so syk_apply_chi, syk_otoc and syk_batch_submit refuse
 *     it; syk_apply_H, syk_krylov_evolve[_noalloc], syk_random_state (block
 *     U) and syk_terms_* accept it with block SYK_BLOCK_U (both block slots
 *     hold the same operator).
 * ---------------------------------------------------------------------------
 */

/*
 * syk_build_pauli_terms — compile H = sum_t h[t] P(x[t], z[t]).
 *   n_qubits : 1 <= n_qubits <= 31.
 *   x, z     : HOST uint32 [T], masks below 2^n_qubits.
 *   h        : HOST double [T], finite.
 *   dtype    : SYK_C64 or SYK_C128.
 * Equal strings are merged and zero sums dropped; the table, pass plan and
 * records are built and uploaded to the current device as for
 * syk_build_terms (T = 0 gives H = 0).  Errors: SYK_EINVAL (n_qubits out of
 * range, a mask with bits at or above n_qubits, non-finite h, null array),
 * SYK_ENOMEM, SYK_ECUDA.
 */
int syk_build_pauli_terms(int n_qubits, int64_t T, const uint32_t* x, const uint32_t* z, const double* h,
                          int dtype, syk_terms_t** out);

/*
 * Host-only compilation of syk_build_pauli_terms (no CUDA call).  Writes up
 * to `capacity` compiled strings into the HOST arrays (any may be NULL) and
 * the count into *n_terms: flip mask, sign mask, coefficient and imag flag
 * in the form (H psi)[m] = sum_t coef[t] (imag ? i : 1) (-1)^{popc(z & m)}
 * psi[m ^ x] — the form syk_terms_export reports for a Pauli handle.
 */
int syk_compile_pauli_host(int n_qubits, int64_t T, const uint32_t* x, const uint32_t* z, const double* h,
                           int64_t capacity, int64_t* n_terms, uint32_t* x_out, uint32_t* z_out, double* coef,
                           uint8_t* imag);

/*
 * syk_apply_pauli — out = P(x, z) psi (coefficient 1) for nstates states of
 * a Pauli handle; psi, out: [nstates][D] device.  out may alias psi exactly
 * when x = 0 (a diagonal string); otherwise they must not overlap.
 * Errors: SYK_EINVAL (not a Pauli handle, mask out of range, null or
 * misaligned pointer, overlap), SYK_ECUDA.
 */
int syk_apply_pauli(const syk_terms_t* h, uint32_t x, uint32_t z, const void* psi, void* out, int64_t nstates,
                    syk_stream_t stream);

/*
 * syk_pauli_otoc — the regularised OTOC of Eq. (2) with the Majoranas
 * replaced by two Pauli strings W = P(w_x, w_z) and V = P(v_x, v_z), on a
 * single state (the supplement's symmetric beta/8 + beta/8 split):
 *   F(t) = <psi| e^{(it-b/8)H} W e^{-(it+b/4)H} V e^{(it-b/4)H} W
 *          e^{-(it+b/4)H} V e^{-bH/8} |psi>,
 *   OTOC(t) = Re mean_s F_s(t) / Re mean_s F_s(0).
 * mode SYK_OTOC_TYPICAL: states from psi_opt (DEVICE [n_states][D], used as
 * given), else syk_random_state(seed, s) block U normalised over its D
 * amplitudes; SYK_OTOC_EXACT_TRACE: all D basis states, F = Tr[...]/D (one
 * row).  t_grid (HOST, non-decreasing), F_raw (HOST [rows][n_t][2]), otoc
 * (HOST [n_t]), p, stats and the blocking behaviour are as for syk_otoc; the
 * call allocates its own device workspace and frees it before returning.
 * F is not normalised: its size grows like e^{beta |E_min|}, and a spin
 * chain's energies are extensive, so complex64 states overflow once
 * beta |E_min| exceeds about 80.  Adding the identity string (x = z = 0) with
 * weight c to H multiplies every F(t) by e^{-beta c} exactly and leaves the
 * OTOC ratio unchanged; c near -E_min keeps the weights in range.
 * Errors: SYK_EINVAL (not a Pauli handle, mask out of range, bad grid, beta,
 * mode or n_states), SYK_ENOMEM, SYK_ENOCONV, SYK_ECUDA.
 */
int syk_pauli_otoc(const syk_terms_t* h, uint32_t w_x, uint32_t w_z, uint32_t v_x, uint32_t v_z, double beta,
                   const double* t_grid, int n_t, int mode, int n_states, uint64_t seed, const void* psi_opt,
                   const syk_krylov_params* p, double* F_raw, double* otoc, syk_krylov_stats* stats,
                   syk_stream_t stream);

/*
 * ---------------------------------------------------------------------------
 * Non-Hermitian sparse SYK, the other model of the paper's outlook:
 * H = sum_t (J_t + i M_t) chi_i chi_j chi_k chi_l (complex couplings, Eq. (1)
 * otherwise unchanged), so H^dag = sum_t (J_t - i M_t) chi chi chi chi.  The
 * handle runs on the same H psi kernels (each term splits into a real-class
 * and an imaginary-class string); syk_krylov_evolve[_noalloc] on a handle
 * with any M_t != 0 uses Arnoldi (full orthogonalisation, classical
 * Gram-Schmidt twice, FP64 Hessenberg matrix, its exponential by scaling
 * and squaring with a [6/6] Pade approximant on the device) with the same
 * substep control as Lanczos; reorth and two_pass are refused for it, and
 * its workspace is larger (syk_krylov_workspace_bytes).  syk_otoc and the
 * batched engine refuse such a handle; use syk_otoc_nonhermitian.
 * ---------------------------------------------------------------------------
 */

/*
 * syk_build_terms_complex — as syk_build_terms with couplings J_re + i J_im
 * (HOST double [T] each).  With J_im all zero the handle equals
 * syk_build_terms(J_re) (Hermitian, Lanczos).  Errors as syk_build_terms.
 */
int syk_build_terms_complex(int N, int64_t T, const int32_t* quads, const double* J_re, const double* J_im, int dtype,
                            int rep, syk_terms_t** out);

/* Host-only compilation of syk_build_terms_complex, in the form of
 * syk_compile_terms_host (no CUDA call). */
int syk_compile_terms_complex_host(int N, int64_t T, const int32_t* quads, const double* J_re, const double* J_im,
                                   int rep, int64_t capacity, int64_t* n_terms, uint32_t* x, uint32_t* z,
                                   double* coef_U, double* coef_D, uint8_t* imag);

/* *hermitian = 1 if the handle's Krylov propagation is Lanczos, 0 if Arnoldi. */
int syk_terms_is_hermitian(const syk_terms_t* h, int* hermitian);

/*
 * syk_terms_adjoint — a new handle for H^dag on the current device (same N,
 * representation, dtype; Pauli handles too).  A block string
 * c (imag ? i : 1) S with S[m, m ^ x] = (-1)^{popc(z & m)} has adjoint
 * conj(c (imag ? i : 1)) (-1)^{popc(x & z)} S.  The caller destroys it.
 */
int syk_terms_adjoint(const syk_terms_t* h, syk_terms_t** out);

/*
 * syk_otoc_nonhermitian — the OTOC of Eq. (2) at infinite temperature with
 * the Heisenberg-picture operator W(t) = e^{iH^dag t} W e^{-iHt} (the paper
 * gives no formula for non-Hermitian H; with M = 0 this is syk_otoc at
 * beta = 0):
 *   F_P(t) = <psi_P| e^{iH^dag t} chi_a e^{-iH_QQ t} chi_b e^{iH^dag_PP t}
 *            chi_a e^{-iH_QQ t} chi_b |psi_P>,  F = F_U + F_D,
 *   OTOC(t) = Re mean_s F_s(t) / Re mean_s F_s(0).
 * Arguments, modes, outputs and blocking as for syk_otoc without beta;
 * H^dag is built internally (syk_terms_adjoint) for the call.  Errors:
 * SYK_EINVAL, SYK_ENOMEM, SYK_ENOCONV, SYK_ECUDA.
 */
int syk_otoc_nonhermitian(const syk_terms_t* h, int a, int b, const double* t_grid, int n_t, int mode, int n_states,
                          uint64_t seed, const void* psi_opt, const syk_krylov_params* p, double* F_raw, double* otoc,
                          syk_krylov_stats* stats, syk_stream_t stream);

/*
 * Batched OTOC engine — many (realisation, state) OTOC curves at once.
 * Each job is the typical-state OTOC of syk_otoc for one Hamiltonian handle
 * (any N, same dtype as the batch), one Philox state (syk_random_state(seed,
 * state_id), normalised over both blocks) and its own beta and time grid.  A
 * job occupies a slot and device memory from the batch's arena
 * ((m + 5) block vectors plus the grid; syk_batch_job_bytes) until it
 * finishes; jobs of different N share every launch.  One tick advances every
 * live job by one Krylov substep; the tick is a captured CUDA graph (Lanczos
 * kernels batched over jobs, a per-job device state machine for the
 * elementwise steps), so the host only admits and collects.  Lanczos uses a
 * stored basis (no two_pass / reorth).
 */
typedef struct syk_batch syk_batch_t;
typedef struct {
  const syk_terms_t* h;      /* Hamiltonian (kept alive by the caller until the job finishes) */
  int a, b;                  /* Majoranas of the OTOC */
  double beta;
  const double* t_grid;      /* HOST [n_t], non-decreasing; copied at submit */
  int n_t;
  uint64_t seed, state_id;   /* typical state */
  int64_t tag;               /* caller's id, reported back when the job finishes */
  double* F_out;             /* HOST [n_t][2] (re, im of F(t)), written when the job finishes */
  syk_krylov_stats* stats;   /* HOST, optional */
  int* status_out;           /* HOST, optional: SYK_OK or SYK_ENOCONV when the job finishes */
  int64_t basis_index;       /* < 0: typical state; else the basis state g = block*D + m of the
                                full space (exact trace = sum of these jobs over g, divided by 2D) */
  int kind;                  /* SYK_JOB_OTOC, or SYK_JOB_GREEN: G(t) = <psi| e^{(it-b/2)H} chi_a
                                e^{-iHt} chi_a e^{-bH/2} |psi> (supplement, Green function; b unused) */
  double* otoc_out;          /* HOST [n_t], optional: the job's normalised curve Re F(t) / Re F(0)
                                (Re G(t) / Re G(0) for SYK_JOB_GREEN), written when it finishes */
} syk_otoc_job;
enum { SYK_JOB_OTOC = 0, SYK_JOB_GREEN = 1 };
/* max_bytes: device arena for job state (allocated once); max_slots: jobs in flight;
 * p: Krylov parameters shared by all jobs (zero fields take the defaults of
 * syk_krylov_params; two_pass and reorth must be 0). */
int syk_batch_create(int dtype, int max_slots, size_t max_bytes, const syk_krylov_params* p, syk_batch_t** out);
int syk_batch_destroy(syk_batch_t* batch);
/* Admit a job; SYK_EAGAIN if no slot or no arena range is free (retry after a run). */
int syk_batch_submit(syk_batch_t* batch, const syk_otoc_job* job);
/*
 * Run ticks on the batch's own stream, synchronising every ticks_per_sync
 * ticks, until at least one job finishes or max_ticks ticks have run.  Writes
 * the finished jobs' outputs, frees their slots and memory, and reports how
 * many finished (and up to max_finished of their tags).  Blocking.
 */
int syk_batch_run(syk_batch_t* batch, int max_ticks, int ticks_per_sync, int* n_finished, int64_t* finished_tags,
                  int max_finished);
int syk_batch_info(const syk_batch_t* batch, int* live_jobs, size_t* bytes_in_use, size_t* bytes_free_max);
/* Device bytes a job needs (0 on bad arguments). */
size_t syk_batch_job_bytes(const syk_batch_t* batch, const syk_terms_t* h, int n_t);

/*
 * syk_otoc_exact_trace_batched — the exact-trace OTOC of Eq. (2) for several
 * Majorana pairs through the batched engine: for each pair (a, b),
 *   F_tr(t) = sum_g F_{e_g}(t) / 2D  over the 2D basis states e_g of both
 *   parity blocks (one batched job per (pair, g), as syk_otoc_job with
 *   basis_index = g),  OTOC(t) = Re F_tr(t) / Re F_tr(0).
 *   pairs    : HOST int32 [n_pairs][2] (a, b).
 *   t_grid   : HOST double [n_t], non-decreasing.
 *   max_slots, max_bytes, p : as for syk_batch_create (jobs live at once,
 *              device arena, Krylov parameters; two_pass / reorth refused).
 *   F_out    : HOST double [n_pairs][n_t][2] (re, im of F_tr), may be NULL.
 *   otoc_out : HOST double [n_pairs][n_t], may be NULL.
 *   stats    : HOST, optional: matvecs and substeps summed over all jobs.
 * The sum over g runs in the fixed order g = 0, 1, ..., 2D-1 in FP64 on the
 * host, whatever order the jobs finish in, so results are reproducible.
 * Blocking; creates and destroys its own batch.  Errors: SYK_EINVAL,
 * SYK_ENOMEM, SYK_ENOCONV (a job did not converge), SYK_ETIMEOUT, SYK_ECUDA.
 */
int syk_otoc_exact_trace_batched(const syk_terms_t* h, int n_pairs, const int32_t* pairs, double beta,
                                 const double* t_grid, int n_t, int max_slots, size_t max_bytes,
                                 const syk_krylov_params* p, double* F_out, double* otoc_out,
                                 syk_krylov_stats* stats);

/*
 * syk_bounded_wait_selftest — failure-detection self-test (no paper
 * counterpart): one CTA waits, with the bounded wait of the TMA pipelines, on
 * an mbarrier that nothing completes.  Returns SYK_ETIMEOUT after the wait
 * limit (~1 s) — the expected outcome — with the context still usable;
 * SYK_ECUDA if the wait did not expire or a CUDA call failed.  Synchronises
 * `stream`.
 */
int syk_bounded_wait_selftest(syk_stream_t stream);

/*
 * syk_relabel_majoranas — a Jordan-Wigner ordering of the Majoranas that
 * lowers the number of distinct flip patterns above the matvec tile, i.e.
 * the input tiles the complex64 H psi stages per output tile (the paper has
 * no counterpart: its representation is Eq. (S1)).  A relabelling of the
 * Majoranas is an automorphism of the Clifford algebra, implemented by a
 * unitary on the state space, so the spectrum of H and the exact-trace OTOC
 * of Eq. (2) do not change; single states are expressed in the new basis.
 *   quads, J   : HOST, as for syk_build_terms (N Majoranas, T terms).
 *   tile_bits  : amplitude bits inside a tile (11 for this library's kernels).
 *   iterations : simulated-annealing moves (swaps of two Majoranas between
 *                qubits; e.g. 200000); seed: the moves' random seed
 *                (deterministic for a given seed).
 *   perm       : HOST int32 [N] out: physical Majorana i becomes Jordan-Wigner
 *                Majorana perm[i]; Majoranas N-2 and N-1 keep the top qubit
 *                (perm[N-2] = N-2, perm[N-1] = N-1), so chi_{N-1}, chi_{N-2}
 *                stay diagonal between the parity blocks.
 *   quads_out, J_out : HOST [T][4], [T] out (may be NULL): the same
 *                Hamiltonian in the new labels, each quadruple sorted and its
 *                coupling multiplied by the sign of the sorting permutation
 *                (distinct Majoranas anticommute); pass them to
 *                syk_build_terms with SYK_REP_JW.
 *   patterns_before / after : HOST, may be NULL: distinct patterns of the
 *                identity ordering and of the returned one.
 * Host-only (no CUDA call).  Errors: SYK_EINVAL.
 */
int syk_relabel_majoranas(int N, int64_t T, const int32_t* quads, const double* J, int tile_bits, int64_t iterations,
                          uint64_t seed, int32_t* perm, int32_t* quads_out, double* J_out, int64_t* patterns_before,
                          int64_t* patterns_after);

/*
 * syk_tridiag_exp — the projected-exponential step of the Krylov engine on a
 * caller's Lanczos matrix (supplement Sec. I.A, the Krylov time evolution;
 * exposed for testing): T = tridiag(beta[0..m-2], alpha[0..m-1],
 * beta[0..m-2]) with residual beta[m-1] (HOST arrays of m; beta >= 0), the
 * largest fraction s = 2^-k of z = z_re + i z_im whose a-posteriori error
 * estimate is <= tol * s, and c = e^{-s z T} e_1.  force_ql = 1 takes the QL
 * eigensolver instead of the lane-parallel one.  Outputs (HOST): c [m][2]
 * (re, im), *s_acc (0 if no fraction passed), *err, *used_ql (1 if the QL
 * path ran; may be NULL), *kernel_ms (may be NULL: then the step is also
 * timed, the median of 5 launches by CUDA events).  Blocking, on the legacy
 * default stream.  Errors: SYK_EINVAL, SYK_ENOMEM, SYK_ENOCONV, SYK_ECUDA.
 */
int syk_tridiag_exp(int m, const double* alpha, const double* beta, double z_re, double z_im, double tol, int force_ql,
                    double* c, double* s_acc, double* err, int* used_ql, double* kernel_ms);

/*
 * Hardware probes for the benchmark's roofline denominators (no paper
 * counterpart; the hot path never calls them).  Each synchronises `stream`.
 *
 * syk_probe_staging — bytes per second moved from `buf` (DEVICE, `bytes`
 * long, 16-byte aligned, at least 16 KiB; make it smaller than L2 to measure
 * L2 -> shared memory) by the pipeline shape of the complex64 matvec's store
 * passes: 16 KiB bulk copies (cp.async.bulk + mbarrier), 2 stages, one
 * producer lane and 4 consumer warps per CTA, 5 CTAs per SM, `jobs_per_cta`
 * tiles per CTA on a
 * scattered walk over the buffer.  reads = 0: the consumers only wait for and
 * release each stage; 1 or 2: they also read every staged tile that many
 * times from shared memory (16-byte loads); -1: no shared memory, the same
 * tiles read with 16-byte global loads that do not allocate in L1.  The rate
 * counts the tile bytes fetched from `buf` once per job.  One warm-up launch,
 * then one timed launch (CUDA events).  Errors: SYK_EINVAL, SYK_ENOMEM,
 * SYK_ETIMEOUT (a bounded wait expired), SYK_ECUDA.
 */
int syk_probe_staging(const void* buf, size_t bytes, int reads, int jobs_per_cta, double* bytes_per_s,
                      syk_stream_t stream);
/* syk_probe_smem — bytes per second of 16-byte shared-memory loads of the
 * whole GPU (8 CTAs of 128 threads per SM, each streaming over a 16 KiB tile
 * in its shared memory; a warp's load covers 512 contiguous bytes, as in the
 * complex64 matvec consumers).  One warm-up launch, one timed launch (CUDA
 * events).  Errors: SYK_EINVAL, SYK_ENOMEM, SYK_ECUDA. */
int syk_probe_smem(double* bytes_per_s, syk_stream_t stream);
/* syk_probe_fp64 — FP64 fused multiply-adds per second of the whole GPU
 * (8 independent chains per thread, 8 CTAs of 256 threads per SM). */
int syk_probe_fp64(double* dfma_per_s, syk_stream_t stream);

/* Message of the last failing call on this thread (always NUL-terminated). */
int syk_last_error(char* buf, size_t n);
/* Library version string. */
const char* syk_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SYK_H */
