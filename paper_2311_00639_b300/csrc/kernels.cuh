// Launchers for the libsyk device kernels (apply.cu, krylov.cu).
#pragma once

#include "internal.h"

namespace syk {

// Counts summed on the device over the evolves that share one workspace (the
// single-realisation Lanczos path keeps its substep control on the device).
struct KTotals {
  long long matvecs, substeps;
  double err;  // sum of accepted local error estimates x accepted fractions
  int fail;    // first failure: 1 no acceptable substep, 2 eigensolver, 3 max_substeps reached
  int ql;      // substeps whose eigensystem came from the QL fallback (tridiag.cuh)
};

// Device-side scalars of one Lanczos run (float64 throughout).
struct KScalars {
  double alpha[kMaxKrylov];
  double beta[kMaxKrylov];  // beta[j] = ||w_j||, the (j, j+1) entry of T; beta[m-1] = residual
  double beta0;             // ||x||
  double c_re[kMaxKrylov], c_im[kMaxKrylov];
  double s_acc;             // accepted fraction of the remaining step
  double err;               // relative local error estimate of the accepted step
  int m_eff;                // basis vectors in use (< m after a breakdown)
  int status;               // 0 ok; 1 no acceptable substep; 2 eigensolver did not converge
  // device-side substep control of one evolve (single-realisation path)
  double z_re, z_im;  // the part of z = tau + i t still to be applied
  double tol;
  int n_sub, max_sub;
  int fail;  // this evolve failed (see KTotals::fail)
  int pad_;
  KTotals tot;
};

inline size_t elem_bytes(int dtype) { return dtype == SYK_C128 ? 16 : 8; }

// Grid used by every streaming vector kernel for a vector of D amplitudes.
int vec_grid(const syk_terms* h);
// Grid.x of the matvec kernel (the number of reduction partials it writes).
int matvec_grid(const syk_terms* h);

// out = H_P psi for nstates contiguous states.
void launch_apply_H(const syk_terms* h, int block, const void* psi, void* out, int64_t nstates,
                    cudaStream_t st);
// out = chi_n psi (block from_block -> other block), nstates states.
void launch_apply_chi(const syk_terms* h, int n, int from_block, const void* psi, void* out,
                      int64_t nstates, cudaStream_t st);
// Philox4x32-10 + Box-Muller amplitudes (unnormalised) of one block.
void launch_random_state(const syk_terms* h, uint64_t seed, uint64_t state_id, int block, void* psi,
                         cudaStream_t st);

// --- Lanczos building blocks (single state, vectors of D amplitudes) ---
// partial[b] = sum |x|^2 over the blocks of vec_grid.
void launch_norm_partials(const syk_terms* h, const void* x, double* partial, cudaStream_t st);
// v0 = x / ||x||, sc->beta0 = ||x||, sc->m_eff = m (0 if x = 0).
void launch_scale_first(const syk_terms* h, const void* x, void* v0, const double* partial, KScalars* sc,
                        int m, cudaStream_t st);
// w = H_P v_j - beta_{j-1} v_{j-1}; partial[b] = Re <v_j, w>.  vprev may be null (j = 0).
void launch_lanczos_matvec(const syk_terms* h, int block, const void* v, const void* vprev, void* w,
                           double* partial, KScalars* sc, int j, cudaStream_t st);
// alpha_j = sum partialA; w -= alpha_j v_j; partialN[b] = sum |w|^2.
void launch_axpy_norm(const syk_terms* h, void* w, const void* v, const double* partialA, int npA,
                      double* partialN, KScalars* sc, int j, cudaStream_t st);
// Full re-orthogonalisation of w against V[0..j] (classical Gram-Schmidt, twice);
// leaves sum |w|^2 partials in partialN.
void launch_reorth(const syk_terms* h, void* w, const void* V, int j, double* partialR, double* partialN,
                   KScalars* sc, cudaStream_t st);
// beta_j = sqrt(sum partialN); v_{j+1} = w / beta_j (in place); breakdown sets m_eff = j+1.
void launch_scale_next(const syk_terms* h, void* w, const double* partialN, int npN, KScalars* sc, int j,
                       double breakdown_abs, cudaStream_t st);
// Eigen-decompose T_m, choose the substep s in (0, 1] of z, write c = e^{-s z T} e_1.
void launch_tridiag(KScalars* sc, int m, double z_re, double z_im, double tol, cudaStream_t st);
// y = beta0 * sum_j c_j V_j (stored basis).
void launch_combine(const syk_terms* h, const void* V, void* y, const KScalars* sc, int m, cudaStream_t st);
// Second pass: v0 = x / beta0; y = beta0 c_0 v0.
void launch_recur_first(const syk_terms* h, const void* x, void* v0, void* y, const KScalars* sc,
                        cudaStream_t st);
// Second pass step j: v_{j+1} = (H v_j - beta_{j-1} v_{j-1} - alpha_j v_j) / beta_j (same rounding
// sequence as the first pass), y += beta0 c_{j+1} v_{j+1}.
void launch_lanczos_recur(const syk_terms* h, int block, const void* v, const void* vprev, void* vnext,
                          void* y, const KScalars* sc, int j, cudaStream_t st);

// --- OTOC helpers ---
// partial[b] = (re, im) of sum conj(a) b.
void launch_zdot_partials(const syk_terms* h, const void* a, const void* b, double* partial, cudaStream_t st);
// out[0..1] (+)= sum of partials (re, im), times `scale`.
void launch_zdot_finalize(const double* partial, int np, double* out, double scale, int accumulate,
                          cudaStream_t st);
// *acc (+)= sum of real partials.
void launch_sum_finalize(const double* partial, int np, double* acc, int accumulate, cudaStream_t st);
// x *= 1/sqrt(*n2).
void launch_scale_inv_sqrt(const syk_terms* h, void* x, const double* n2, cudaStream_t st);
// x = e_k (unit vector) or zero.
void launch_basis_vector(const syk_terms* h, void* x, int64_t k, cudaStream_t st);

// --- Krylov engine (krylov.cu) ---
struct KrylovResult {
  int64_t matvecs = 0, substeps = 0;
  double err = 0.0;
};
// The Lanczos path of krylov_evolve_one queues its work and counts on the
// device (KScalars::tot of the workspace): reset the totals before a sequence
// of evolves that share a workspace, and collect them after it (collect
// synchronises the stream, adds the counts to `acc` and throws SYK_ENOCONV if
// an evolve failed).  The Arnoldi path still returns its counts directly.
void krylov_totals_reset(void* ws, cudaStream_t st);
void krylov_totals_collect(void* ws, cudaStream_t st, KrylovResult& acc);
size_t krylov_ws_bytes(const syk_terms* h, int m, bool two_pass);
// Arnoldi engine for a non-Hermitian H (arnoldi.cu); krylov_* dispatch to it
// when h->hermitian is false.
size_t arnoldi_ws_bytes(const syk_terms* h, int m);
KrylovResult arnoldi_evolve_one(const syk_terms* h, int block, double tau, double t, const void* x, void* y, int m,
                                double tol, int max_substeps, void* ws, cudaStream_t st);
// y = e^{-(tau + i t) H_P} x for one state; y may alias x.
KrylovResult krylov_evolve_one(const syk_terms* h, int block, double tau, double t, const void* x, void* y, int m,
                               double tol, int max_substeps, bool reorth, bool two_pass, void* ws, cudaStream_t st);

}  // namespace syk
