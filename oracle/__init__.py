"""CPU oracle for the unfitted BAE method with lattice Green's functions.

TEST INFRASTRUCTURE ONLY. Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import anything in this package. The
library in `paper_2502_05507_gb300/` never imports it, shares no code with it,
and fails loudly when its CUDA extension is missing instead of falling back
here.

Everything is plain numpy/scipy in float64, written from the paper
(Xia, "Unfitted boundary algebraic equation method based on difference
potentials and lattice Green's function in 3D"):

  grid.py        point sets M+, M-, N+, gamma+-, D_n (Section 2.1) and the
                 Dirichlet closure on grid edges (eq. [bc])
  lgf.py         lattice Green's function by Watson's Bessel integral
                 (eq. [lgf_bessel]) and its far-field expansion (Section 2.2)
  potentials.py  single/double-layer potentials by direct summation
                 (Section 3.2, eqs. [single], [single_potential],
                 [double_potential]), particular solution, and the
                 same convolutions by a plain zero-padded FFT
  gmres.py       unrestarted GMRES with modified Gram-Schmidt
  fd.py          the discrete problem assembled as a sparse finite-difference
                 system (eq. [discrete] plus the closure rows), solved directly
  solve.py       Algorithm 1 end to end (double or single layer)
  direct.py      the direct formulation: unknown u on gamma, difference
                 potentials P w = G_h[chi_{M-} L_h w] (eqs. [dp], [bep],
                 [direct_sys], [discrete_green])

Equations are cited by their LaTeX labels in brackets, e.g. eq. [lgf].
Parity status per function is listed in each module header.
"""
