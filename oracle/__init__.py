"""FP64 CPU oracle for non-Hermitian FEAST / Bi-FEAST (Tang, Kestyn & Polizzi).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code with the CUDA library.

Everything here is plain, slow and written to be checked against the paper by
eye: complex128 throughout, its own Gaussian elimination with partial pivoting
and its own triangular solves, the quadrature of Sec. 3, the filter of
Eq. Rasp / Eq. Lasp and the two subspace iterations of Sec. 4.  Library
routines appear only as single steps (a matrix product, ``scipy.linalg.eig`` for
the small reduced pencil and for the brute-force reference spectrum).

Modules
-------
contour   -- Eq. ellipses, Eq. pi, Eq. quadrature_for_pi: nodes phi_k, weights sigma_k
dense     -- Gaussian elimination with partial pivoting and the two solves
feast     -- Eq. Rasp, Eq. Lasp, Algorithms R-FEAST and Bi-FEAST, Sec. 5 monitoring
brute     -- the plain definition: every eigenpair of (A, B), filtered to the domain
moments   -- stochastic estimate of tr rho(M) and its higher moments (count estimation, Sec. 6)
mlp       -- the small count-predictor network: forward, backward, Adam, in FP64

Parity unpinned: none of the functions above is unpinned; the exact pivot
sequence of a low-precision factorisation is not an oracle output.
"""
