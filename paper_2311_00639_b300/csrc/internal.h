// Internal declarations shared by the libsyk translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "syk.h"

namespace syk {

constexpr int kMaxKrylov = 64;   // largest Krylov dimension per substep
constexpr int kTileBits = 11;    // amplitudes per matvec tile = 2^11 (one 16 KiB complex64 bulk copy)
constexpr int kMaxPartials = 2048;  // per-state reduction partials (>= any grid.x)

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define SYK_CUDA(expr)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      throw ::syk::Error(SYK_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));    \
  } while (0)
#define SYK_REQUIRE(cond, msg)                                   \
  do {                                                           \
    if (!(cond)) throw ::syk::Error(SYK_EINVAL, (msg));          \
  } while (0)

// One Pauli string acting inside a parity block (block-compressed form):
//   (O psi)[m] = coef[P] * (imag ? i : 1) * (-1)^{popc(z & m)} * psi[m ^ x].
struct BlockString {
  uint32_t x = 0, z = 0;
  double coef[2] = {0.0, 0.0};  // block U, block D
  bool imag = false;
  bool straggler = false;  // read from outside its pass's L2-resident super-tile
};

// A single Majorana restricted to block P -> 1-P, same output-index form,
// with a complex coefficient per source block (chi = gamma / sqrt 2 included).
struct ChiString {
  uint32_t x = 0, z = 0;
  double re[2] = {0, 0}, im[2] = {0, 0};
};

// Term compiler (terms.cpp).
void compile_terms(int N, int rep, int64_t T, const int32_t* quads, const double* J,
                   std::vector<BlockString>& out, int64_t& n_real, int64_t& n_xgroups);
ChiString compile_chi(int N, int rep, int n);
// Complex couplings J_re + i J_im (non-Hermitian SYK): each term's value
// splits into a real-class and an imaginary-class string with the same masks.
void compile_terms_complex(int N, int rep, int64_t T, const int32_t* quads, const double* J_re, const double* J_im,
                           std::vector<BlockString>& out, int64_t& n_real, int64_t& n_xgroups);

// Record the message syk_last_error() returns on this thread (capi.cu).
void set_last_error(const std::string& msg);

// One pass of the blocked matvec (plan.cpp).  Terms [t0, ti) have a real
// coefficient and [ti, t1) an imaginary one; tile index bt maps to the first
// amplitude dep[0][bt & 255] | dep[1][(bt >> 8) & 255] | dep[2][(bt >> 16) & 255].
// The same struct is copied to the device.
struct PassPlan {
  int t0 = 0, ti = 0, t1 = 0;
  uint32_t emask = 0;  // bits held fixed within a super-tile
  // Terms of class c = 4*imag + 2*(x & 1) + (z & 1) are [cls[c], cls[c+1]).
  int cls[9] = {};
  uint32_t dep[3][256] = {};
};
// Packed complex64 term record (one 16-byte load per term).  The complex64
// record array keeps each pass's terms together but orders them inside the
// pass by (x >> kTileBits, class, x, z), so that the terms that read the same
// input tile (a "run") are adjacent and share one staged copy of it.
struct alignas(16) TermF {
  uint32_t x, z;
  float c;
  uint32_t flags;
};
constexpr uint32_t kTermStraggler = 1u;  // the run's input tiles come from HBM (fetched evict-first)
constexpr uint32_t kTermRunStart = 2u;   // first term of a run: a new input tile
constexpr uint32_t kTermRunEnd = 4u;     // last term of a run: its stage is released after it
constexpr uint32_t kTermImag = 8u;       // coefficient i * c
// The next record of the pass has the same flip mask x and the same class
// (imag, z & 1), so the same consumer body on the same staged inputs: the
// consumer adds this term's signed row coefficients to a running sum and
// applies the body once, with the sum, at the last term of such a group
// (dense SYK: many strings share x; x and class equal implies the same run).
constexpr uint32_t kTermMerge = 16u;
// Bits 16-23 of a merge group's first record: how many records follow it in
// the group (groups longer than 256 records are split into groups of at most
// 256), so that the consumer sums the group in one tight loop.
constexpr int kTermGroupShift = 16;
constexpr uint32_t kTermGroupMax = 255u;
// Bits 8-13 of flags: the consumer body of the term, 32 imag + 16 (x & 1) +
// 8 (z & 1) + ((x >> 6) & 7) (class and row permutation of the 8-row layout).
// Bit 31 of flags, x and z (x and z use at most 31 bits) hold z's bits 6, 7
// and 8: the sign pattern of the 8 rows, so that the consumer forms each
// row's signed coefficient with one masked XOR.  Readers of x for addresses
// use kTermXMask.
constexpr uint32_t kTermXMask = 0x7FFFFFFFu;
constexpr int kTermBodyShift = 8;
inline uint32_t term_body(uint32_t x, uint32_t z, bool imag) {
  return (imag ? 32u : 0u) | ((x & 1u) << 4) | ((z & 1u) << 3) | ((x >> 6) & 7u);
}
// Chooses the term split of each complex64 pass (apply.cu).
void plan_split(syk_terms* h);
// Complex64 records of both blocks in the kernel's order, n + 1 per block (the
// last one zero); returns the number of runs (records.cpp).
int64_t build_records(const std::vector<BlockString>& terms, const std::vector<PassPlan>& passes,
                      std::vector<TermF> rec[2], int64_t* n_merges = nullptr);
// The last pass's tile order with no terms (the epilogue after a split pass).
PassPlan tail_pass(const PassPlan& last);
// Reorders `terms` by pass and returns the passes.
std::vector<PassPlan> plan_passes(std::vector<BlockString>& terms, int L, size_t elem_bytes, size_t l2_budget,
                                   double hbm_ratio);
// Default pass plan per dtype: the best of B300 budget x ratio sweeps at
// N = 64.  complex64 passes draw their tiles from a shared counter, so every
// CTA stays inside the same super-tiles and large (L2/4) super-tiles stay
// resident; complex128 passes split tiles statically and are FP64-bound, so
// they keep small super-tiles.
inline size_t default_l2_budget(int dtype) { return dtype == SYK_C64 ? size_t(32) << 20 : size_t(2) << 20; }
inline double default_hbm_ratio(int dtype) { return dtype == SYK_C64 ? 3.0 : 1.5; }
// Default Krylov dimension per substep: the fastest OTOC curves on B300
// (complex64, N=30: m=20 176 ms, m=30 227 ms; complex128 at its 1e-12
// tolerance: m=30 260 ms, m=20 291 ms).
inline int default_krylov_m(int dtype) { return dtype == SYK_C64 ? 20 : 30; }

// Device view of a compiled term table, in compute precision Real.
template <typename Real>
struct TermsView {
  const uint32_t* x;
  const uint32_t* z;
  const Real* coef;  // coefficients of the block being applied
};

// A captured single-realisation Krylov evolve: one substep as the body of a
// CUDA-graph while-loop whose condition the tridiagonal step sets, for one
// (block, output vector, workspace, m, reorth, two_pass).
struct KrylovGraph {
  int block = 0;
  const void* y = nullptr;
  const void* ws = nullptr;
  int m = 0;
  bool reorth = false, two_pass = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t used = 0;
};

}  // namespace syk

struct syk_terms {
  int N = 0, L = 0, dtype = 0, rep = 0, device = 0;
  int64_t D = 0, n_input = 0, n_real = 0, n_xgroups = 0;
  double sum_abs = 0.0;
  std::vector<syk::BlockString> terms;
  syk::ChiString chi[64];
  // Device table: x[n], z[n], coef[2][n] in the dtype's precision.
  void* d_mem = nullptr;
  uint32_t* d_x = nullptr;
  uint32_t* d_z = nullptr;
  void* d_coef[2] = {nullptr, nullptr};
  std::vector<syk::PassPlan> passes;
  syk::PassPlan* d_passes = nullptr;
  syk::TermF* d_termf[2] = {nullptr, nullptr};  // complex64 handles: packed terms per block
  int* d_err = nullptr;  // set by a kernel whose bounded wait expired
  unsigned long long* d_sched = nullptr;  // complex64 matvec tile counter pair (zero between launches)
  uint32_t* d_zi = nullptr;  // z | (imag << 31) per term (batched engine)
  int64_t n_runs = 0;  // complex64 record runs (input tiles staged per output tile, all passes)
  int64_t n_merges = 0;  // complex64 records flagged kTermMerge
  // The merging complex64 kernels (their running sums cost registers and the
  // 2 x 5 shape) pay when at least half of the terms merge into groups (dense
  // SYK: 84 %); sparse Hamiltonians merge a term or two and keep the others.
  bool c64_merge() const { return 2 * n_merges >= static_cast<int64_t>(terms.size()) && n_merges > 0; }
  // Store passes run 2 stages x 5 CTAs per SM when runs are short (sparse SYK
  // at N=64: 1.9 terms per staged tile, the spin chain at L=31: 5.6; more
  // consumer warps hide more latency) and 3 x 4 when runs are long (16 or
  // more terms per staged tile) or terms merge (dense SYK: each warp's own
  // load-level parallelism, with 96 registers, matters more).
  bool c64_wide() const { return c64_merge() || static_cast<int64_t>(terms.size()) >= 16 * std::max<int64_t>(n_runs, 1); }
  // complex64 passes of a small block with many terms are split into chunks of
  // terms applied by different CTAs (plan_split): chunks per pass (1 = not
  // split) and terms per chunk; partial sums go to d_split_ws.
  std::vector<int> split_chunks, split_terms;
  float2* d_split_ws = nullptr;
  size_t split_ws_bytes = 0;
  syk::PassPlan* d_pass_tail = nullptr;  // the last pass's tile order with no terms (epilogue after a split)
  int n_sm = 148;
  bool hermitian = true;  // false: complex couplings; Krylov propagation uses Arnoldi
  // captured Krylov evolves (krylov.cu), least recently used dropped first;
  // cleared whenever the device table is re-uploaded
  mutable std::vector<syk::KrylovGraph> kgraphs;
  mutable cudaStream_t cap_stream = nullptr;
  mutable uint64_t kg_clock = 0;
  void clear_graphs() const {
    for (auto& g : kgraphs) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.graph) cudaGraphDestroy(g.graph);
    }
    kgraphs.clear();
  }
  syk_terms() = default;
  syk_terms(const syk_terms&) = delete;
  syk_terms& operator=(const syk_terms&) = delete;
  ~syk_terms() {
    if (!kgraphs.empty()) cudaDeviceSynchronize();
    clear_graphs();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (d_mem) cudaFree(d_mem);
    if (d_split_ws) cudaFree(d_split_ws);
  }
};
