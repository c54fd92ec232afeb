"""Plain, slow FP64 CPU oracle of the FFT-accelerated multi-block Poisson solve (Costa, arXiv 2106.03583).

TEST INFRASTRUCTURE ONLY. The only code allowed to import, call or execute anything in this package is
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg. The CUDA
product path never touches it, and it shares no code with the CUDA library: the two only read the
same seeded inputs (``paper_2106_03583_gb300.inputs``).

What it computes, in the paper's order (Algorithm 1, Sec. 2):
  * ``transforms``: the real-to-real transforms of Table 1 as O(n^2) direct sums, their inverses
    scaled by the normalisation theta, and the eigenvalues lambda_q;
  * ``grid``: the second-order finite-volume operator of Eq. 8 on a stretched multi-block grid,
    assembled as sparse matrices from the staggered ghost-cell rules;
  * ``mg``: a textbook cell-centred geometric multigrid V-cycle for the reduced 2-D equation
    (Eq. 9), red-black Gauss-Seidel, dense direct solve on the coarsest level;
  * ``solve``: forward transform, one multigrid solve per wavenumber, inverse transform; plus a
    dense direct solve of the whole 3-D system for tiny grids.

Pins (tests/test_oracle_*.py): library transforms (scipy.fft), round trips x theta, closed-form
eigenvalues of every boundary-condition pair, manufactured eigenfunction solutions, a triple-transform
closed-form solve on uniform boxes, the factorisation of the operator into the staggered divergence of
the staggered gradient, volume-weighted symmetry, dense LU on tiny grids, the zero-mean invariant and
partition invariance; for the multigrid pieces one at a time: restriction moments, exactness of the
prolongation on affine fields (with the face ghosts), exact colour half-sweeps, coarse operators
equal to the direct assembly on every other face, and a grid-independent V-cycle contraction.
No function here is "parity unpinned".
"""
