"""CPU oracle for the nested-grid Poisson / 2LPT / gradient path (float64, numpy).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import this package.  It shares no code with the CUDA
library: stencil tables, interpolation weights and every step of the method
are written here independently from Hahn & Abel 2011 (arXiv:1103.6031):

* stencils.py   - Table 1 (FD Laplacian / gradient and their Fourier symbols),
                  Table 2 (face-flux operators), Lagrange weights.
* fft_solve.py  - exact DFT solve of the discrete periodic operator (the plain
                  definition that a single-level solve must reach).
* hierarchy.py  - levels, ghost zones, coarse-fine interpolation and flux
                  matching (Sec. 3.3), restriction and injection (Sec. 3.2).
* multigrid.py  - the FAS V-cycle of Sec. 3.2 extended to nests (Sec. 3.3).
* lpt.py        - 2LPT source tau (Sec. 3.1.2) and the -grad phi displacement
                  (eq. of Sec. 3.1.1), each with finite differences of Table 1.

Parity status: single-level results are pinned to closed forms and to the
exact DFT solve; the composite (nested) solve is pinned by invariants only
(flux telescoping, conservation, zero mean, convergence rate, the degraded
unigrid comparison).  The exact coarse-fine interpolation and flux-correction
choices where the paper is silent are "parity unpinned" beyond those
invariants; the oracle's definition is the contract.
"""
