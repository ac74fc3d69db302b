"""CPU oracle for the sparse-SYK OTOC path — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The product
path (the CUDA library and its Python binding) never calls it and shares no
code with it; the only common module is ``syk_inputs`` (seeded input
generators, none of the method's arithmetic).

Everything here is plain numpy/scipy in float64 / complex128, written from the
paper (arXiv 2311.00639) for obviousness, not speed:

* ``majorana``    dense Majorana matrices from Kronecker products of Pauli
                  matrices (supplement Eq. (S1) and its compact form; the
                  standard Jordan-Wigner form), plus per-basis-state action
                  maps built from the single-site Pauli rules;
* ``hamiltonian`` H = sum_t J_t chi_i chi_j chi_k chi_l (Eq. (1)) as a dense
                  matrix, its parity blocks, a CSR form and sampled rows;
* ``pauli``       the paper's <bits, coeff> encoding and Algorithm 1;
* ``dynamics``    exact e^{-zH} by eigendecomposition and by
                  scipy's expm_multiply;
* ``otoc``        the regularised OTOC of Eq. (2) as an exact trace and as a
                  single-state expectation (full space and parity blocks);
* ``spin``        Pauli-string (spin-chain) Hamiltonians of the paper's
                  outlook: dense Kronecker products, basis-state maps, CSR
                  and sampled rows; their OTOC is ``otoc`` with W, V given
                  as matrices;
* ``nonherm``     non-Hermitian sparse SYK (complex couplings), the other
                  model of the outlook: dense / CSR matrices, scipy expm
                  evolution, and the infinite-temperature OTOC with
                  W(t) = e^{iH^dag t} W e^{-iHt}.

Conventions (shared as a written spec with the CUDA side, not as code):
  qubit s <-> bit s of the basis index; operators are Kronecker products
  op_{q-1} (x) ... (x) op_0; sigma_y = [[0,-i],[i,0]]; chi = gamma/sqrt(2),
  {chi_i, chi_j} = delta_ij.
  Representation "paper": q = N/2 qubits, top qubit = parity block bit
  (0 = U, 1 = D); gamma_n = sigma_x(top) (x) A_n for n <= N-2 with A_n the
  compact form of Eq. (S1); gamma_{N-1} = sigma_y(top) (x) 1.
  Representation "jw": gamma_{2s} = Z_0..Z_{s-1} X_s,
  gamma_{2s+1} = Z_0..Z_{s-1} Y_s; block U = even popcount of the full index,
  D = odd; the block index m drops the top qubit.

Parity status: every function here is pinned by tests in
``tests/test_oracle.py``, ``tests/test_oracle_spin.py`` and
``tests/test_oracle_nonherm.py`` (closed forms, algebraic identities, brute force and
library special cases); none is "parity unpinned".
"""
